"""Failure paths of the C ABI, made on the host: NaN / infinite inputs and a bounded
device wait that gives up.

No test here faults, traps or hangs the GPU.  A wait is made to run out by setting its
bound to zero rounds through gbi_set_wait_limit (every stage wait of the tiled pair
passes then gives up at once); the pass records that on the device, waits with the
default bound for the copies it has in flight and returns, and the host reports
GBI_ERR_TIMEOUT.  Afterwards the same context must solve normally.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle import dynamics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gbi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_0278_gb300 as g
    g.lib()
    return g


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _inputs(N, trunc, seed):
    c = workloads.small_cloud(N, seed, phi=0.05)
    inp = dynamics.trap_inputs(c["R"], c["p"], dict(k=0.01, vs=0.1, s0=0.05, d0=0.02), trunc)
    return c["R"], inp


def _solve(ctx, prm, R, inp, **kw):
    t = {k: dev(v) for k, v in inp.items()}
    return ctx.solve(prm, dev(R), t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"], **kw)


@pytest.mark.parametrize("name,where", [("R", (3, 1)), ("VH", (5, 2)), ("Fe", (0, 0)), ("Te", (7, 2)),
                                        ("Va", (2, 1)), ("Oa", (9, 0))])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_input_is_rejected(gbi, name, where, bad):
    """gbi_solve returns GBI_ERR_ARG for a NaN or infinite entry in any input array, and
    the next solve with finite inputs on the same context is unaffected."""
    R, inp = _inputs(24, 2, 5)
    prm = gbi.params(a=1.0, eta=workloads.ETA_DEFAULT, trunc=2, precision=3, rtol=1e-10, max_iter=200)
    ctx = gbi.Context(0)
    V0, O0, _, _, st0 = _solve(ctx, prm, R, inp)
    assert st0 == gbi.GBI_OK
    R2 = R.copy()
    inp2 = {k: v.copy() for k, v in inp.items()}
    (R2 if name == "R" else inp2[name])[where] = bad
    with pytest.raises(gbi.GbiError) as ei:
        _solve(ctx, prm, R2, inp2)
    assert ei.value.status == gbi.GBI_ERR_ARG
    V1, O1, _, _, st1 = _solve(ctx, prm, R, inp)
    assert st1 == gbi.GBI_OK
    assert torch.equal(V0, V1) and torch.equal(O0, O1)
    ctx.close()


def test_nonfinite_input_in_replayed_solve_graph(gbi):
    """The same check when the solve runs as one replayed CUDA graph: the device guard
    stops every system and the host reports GBI_ERR_ARG."""
    R, inp = _inputs(40, 2, 6)
    prm = gbi.params(a=1.0, eta=workloads.ETA_DEFAULT, trunc=2, precision=3, rtol=1e-10)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gbi.Context(0, stream=stream)
        t = {k: dev(v) for k, v in inp.items()}
        Rd = dev(R)
        outs = [ctx.solve(prm, Rd, t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"]) for _ in range(3)]
        stream.synchronize()
        assert ctx.solve_graph_replays() >= 1
        t["Fe"][4, 1] = float("nan")
        with pytest.raises(gbi.GbiError) as ei:
            ctx.solve(prm, Rd, t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"])
        assert ei.value.status == gbi.GBI_ERR_ARG
        t["Fe"][4, 1] = float(inp["Fe"][4, 1])
        V, O, _, _, st = ctx.solve(prm, Rd, t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"])
        stream.synchronize()
        assert st == gbi.GBI_OK
        assert torch.equal(V, outs[-1][0]) and torch.equal(O, outs[-1][1])
        ctx.close()


def test_solve_host_rejects_nonfinite_input(gbi):
    R, inp = _inputs(16, 2, 7)
    prm = gbi.params(a=1.0, eta=workloads.ETA_DEFAULT, trunc=2, precision=1, rtol=1e-10)
    ctx = gbi.Context(0)
    N = len(R)
    V = np.zeros((N, 3))
    Om = np.zeros((N, 3))
    QH = np.zeros((N, 8))
    inp["VH"][3, 4] = np.nan
    with pytest.raises(gbi.GbiError) as ei:
        ctx.solve_host(prm, R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"], V, Om, QH)
    assert ei.value.status == gbi.GBI_ERR_ARG
    ctx.close()


@pytest.mark.parametrize("precision", [1, 2, 3])
def test_stage_wait_gives_up_and_context_recovers(gbi, precision):
    """Tiled pair passes with a zero wait bound: every stage wait gives up, the solve
    returns GBI_ERR_TIMEOUT, and with the default bound restored the same context gives
    the result of a fresh context."""
    R, inp = _inputs(100, 3, 8)
    prm = gbi.params(a=1.0, eta=workloads.ETA_DEFAULT, trunc=3, precision=precision, rtol=1e-10, max_iter=60,
                     max_refine=3)
    ref_ctx = gbi.Context(0)
    ref_ctx.set_wpt(1)
    Vr, Or, _, _, st = _solve(ref_ctx, prm, R, inp)
    assert st == gbi.GBI_OK
    ref_ctx.close()
    ctx = gbi.Context(0)
    ctx.set_wpt(1)
    ctx.set_wait_limit(0)
    with pytest.raises(gbi.GbiError) as ei:
        _solve(ctx, prm, R, inp, allow_not_converged=True)
    assert ei.value.status == gbi.GBI_ERR_TIMEOUT
    ctx.set_wait_limit(-1)
    V, O, _, _, st = _solve(ctx, prm, R, inp)
    assert st == gbi.GBI_OK
    assert torch.equal(V, Vr) and torch.equal(O, Or)
    # a pass outside a solve: gbi_apply, then gbi_pass_status reports it once
    x = dev(np.random.default_rng(1).normal(size=(25, 100)))
    y = torch.zeros_like(x)
    ctx.set_wait_limit(0)
    ctx.apply(100, 3, 1.0, 2, 2, 1, dev(R), x, y, 1.0, 0.0, True)
    assert ctx.pass_status() == gbi.GBI_ERR_TIMEOUT
    assert ctx.pass_status() == gbi.GBI_OK
    ctx.set_wait_limit(-1)
    ctx.apply(100, 3, 1.0, 2, 2, 1, dev(R), x, y, 1.0, 0.0, True)
    assert ctx.pass_status() == gbi.GBI_OK
    ctx.close()


def test_wait_limit_arguments(gbi):
    ctx = gbi.Context(0)
    with pytest.raises(gbi.GbiError):
        ctx.set_wait_limit(-2)
    ctx.set_wait_limit(5)
    ctx.set_wait_limit(-1)
    ctx.close()
