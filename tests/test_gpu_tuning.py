"""Warps-per-target variants of the FP32 / double-float pair kernel, and the tuner.

Every variant sums the same pairs in a different (fixed) order, so each must meet
the same bound against the FP64 oracle; the tuner only picks among them.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle import galerkin, tensors

pytestmark = pytest.mark.gpu

TOLS = {1: 1e-5, 2: 1e-11}


@pytest.fixture(scope="module")
def gbi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_0278_gb300 as g
    g.lib()
    return g


@pytest.fixture()
def ctx(gbi):
    c = gbi.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def relerr(x, ref):
    return np.abs(np.asarray(x) - ref).max() / max(np.abs(ref).max(), 1e-300)


def _sl(code, d):
    return slice(0, d) if code == 0 else (slice(0, 6) if code == 1 else slice(6, d))


_A = {}


def _case(N, trunc, seed):
    key = (N, trunc, seed)
    if key not in _A:
        s = workloads.small_cloud(N, seed, phi=0.05)
        A = galerkin.assemble(s["R"], 1.0, trunc)
        d = tensors.ModeBasis(trunc).d
        A4 = A.reshape(N, d, N, d).copy()
        for i in range(N):
            A4[i, :, i, :] = 0.0
        _A[key] = (s["R"], A4, d)
    return _A[key]


@pytest.mark.parametrize("trunc,N", [(2, 333), (3, 150), (4, 61)])
@pytest.mark.parametrize("rows,cols", [(2, 2), (2, 1), (1, 0)])
@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("wpt", [1, 2, 3, 4, 8, 16])
def test_every_wpt_matches_oracle(ctx, gbi, trunc, N, rows, cols, precision, wpt):
    R, A4, d = _case(N, trunc, 70 + trunc)
    g = galerkin.self_scalars(trunc, 1.0)
    rs, cs = _sl(rows, d), _sl(cols, d)
    nc = len(range(d)[cs])
    nr = len(range(d)[rs])
    rng = np.random.default_rng(wpt)
    x = rng.normal(size=(nc, N))
    y0 = rng.normal(size=(nr, N))
    add_self = rows == cols or (rows == 1 and cols == 0)
    ref = np.einsum("npmq,qm->pn", A4[:, rs, :, cs], x)
    if add_self:
        off = 0 if cols == 0 else 6
        ref = ref + g[rs][:, None] * x[(range(d)[rs].start - off):(range(d)[rs].stop - off)]
    ref = 1.3 * ref + 0.5 * y0
    ctx.set_wpt(wpt)
    used = ctx.pass_wpt(trunc, rows, cols, precision, N)
    assert used == (wpt if wpt in (1, 3) else min(wpt, 8 if (trunc == 4 or precision == 2) else 16))
    yd = dev(y0)
    ctx.apply(N, trunc, 1.0, rows, cols, precision, dev(R), dev(x), yd, 1.3, 0.5, add_self)
    torch.cuda.synchronize()
    err = relerr(yd.cpu().numpy(), ref)
    assert err < TOLS[precision], err


def test_tune_picks_valid_choices_and_keeps_results(ctx, gbi):
    c = workloads.config1()
    N, trunc = len(c["R"]), c["trunc"]
    prm = gbi.params(a=c["a"], eta=c["eta"], trunc=trunc, precision=2, rtol=1e-10, restart=40, inner_rtol=1e-5)
    R = dev(c["R"])
    p = dev(c["p"])
    inp = ctx.trap_inputs(N, trunc, c["k"], c["vs"], c["s0"], c["d0"], R, p)
    args = (inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
    V0, O0, _, i0, _ = ctx.solve(prm, R, *args)
    V0, O0 = V0.cpu().numpy(), O0.cpu().numpy()
    chosen = ctx.tune(trunc, [0, N], reps=2)
    assert len(chosen) == 6
    fp32_cap = 8 if trunc == 4 else 16
    assert chosen[0] in (1, 2, 3, 4, 8, 16) and chosen[0] <= fp32_cap
    assert all(w in (1, 2, 3, 4, 8) for w in chosen[1:4])
    assert all(w in (1, 2, 3, 4, 8, 16) and w <= fp32_cap for w in chosen[4:])
    assert ctx.pass_wpt(trunc, 2, 2, 1, N) == chosen[0]
    assert ctx.pass_wpt(trunc, 2, 2, 2, N) == chosen[1]
    assert ctx.pass_wpt(trunc, 2, 1, 2, N) == chosen[2]
    assert ctx.pass_wpt(trunc, 1, 0, 2, N) == chosen[3]
    assert ctx.pass_wpt(trunc, 2, 1, 1, N) == chosen[4]
    assert ctx.pass_wpt(trunc, 1, 0, 1, N) == chosen[5]
    assert ctx.pass_wpt(trunc, 2, 2, 0, N) == 0
    V1, O1, _, i1, _ = ctx.solve(prm, R, *args)
    assert i1.rel_residual <= 1e-10
    assert relerr(V1.cpu().numpy(), V0) < 1e-9
    assert relerr(O1.cpu().numpy(), O0) < 1e-9


def test_tune_batched_layout(ctx, gbi):
    sizes = [40, 7, 90, 33]
    offs = [0]
    for n in sizes:
        offs.append(offs[-1] + n)
    chosen = ctx.tune(2, offs, reps=1)
    assert len(chosen) == 6 and all(w in (2, 4, 8, 16) for w in chosen)
    assert ctx.pass_wpt(2, 2, 2, 1, offs[-1], batched=True) == chosen[0]


def test_tune_rejects_bad_layouts(ctx, gbi):
    for offs in ([1, 5], [0, 5, 5], [0]):
        with pytest.raises(gbi.GbiError):
            ctx.tune(2, offs)
    with pytest.raises(gbi.GbiError):
        ctx.set_wpt(5)


@pytest.mark.parametrize("trunc,N", [(2, 2), (2, 33), (3, 64), (3, 97), (2, 1024), (3, 517), (3, 1300),
                                     (4, 203)])
@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("form", [1, 3])
def test_tiled_form_partitions(ctx, gbi, trunc, N, precision, form):
    """The balanced forms split their units evenly over the grid -- (group of 32 targets,
    source) units over blocks for the tiled form (1), (target, 32-source chunk) units over
    warps for the chunk-balanced form (3); whatever the number of groups or chunks,
    partial groups and ranges that cross them, each sums the same pairs as the streaming
    form (to rounding) on three launches in a row (its arrival counters must be back at
    zero after each)."""
    s = workloads.small_cloud(N, 90 + N, phi=0.05)
    R = dev(s["R"])
    d = tensors.ModeBasis(trunc).d
    h = d - 6
    rng = np.random.default_rng(N)
    x = dev(rng.normal(size=(h, N)))
    ctx.set_wpt(4)
    y_ref = torch.zeros((h, N), dtype=torch.float64, device="cuda")
    ctx.apply(N, trunc, 1.0, 2, 2, precision, R, x, y_ref, 1.0, 0.0, True)
    ctx.set_wpt(form)
    assert ctx.pass_wpt(trunc, 2, 2, precision, N) == form
    for _ in range(3):
        y = torch.full((h, N), 7.0, dtype=torch.float64, device="cuda")
        ctx.apply(N, trunc, 1.0, 2, 2, precision, R, x, y, 1.0, 0.0, True)
        torch.cuda.synchronize()
        assert relerr(y.cpu().numpy(), y_ref.cpu().numpy()) < (2e-6 if precision == 1 else 1e-12)
    ctx.set_wpt(0)


@pytest.mark.parametrize("form", [1, 3])
def test_tiled_form_full_size_sampled_rows(ctx, gbi, form):
    """N = 1024 at l <= 3 (the solve workload), FP32 H/H pass in the tiled (1) and the
    chunk-balanced (3) form, against the oracle's dense pair blocks for sampled targets."""
    c = workloads.config2()
    R = c["R"]
    N, trunc = len(R), 3
    d = tensors.ModeBasis(trunc).d
    h = d - 6
    rng = np.random.default_rng(5)
    x = rng.normal(size=(h, N))
    ctx.set_wpt(form)
    y = torch.zeros((h, N), dtype=torch.float64, device="cuda")
    ctx.apply(N, trunc, c["a"], 2, 2, 1, dev(R), dev(x), y, 1.0, 0.0, False)
    torch.cuda.synchronize()
    ctx.set_wpt(0)
    tg = np.array([0, 31, 32, 511, 700, 1023])
    xf = np.zeros((N, d))
    xf[:, 6:] = x.T
    ref = galerkin.apply_offdiag(R, xf, c["a"], trunc, rows=slice(6, d), targets=tg)
    got = y.cpu().numpy()[:, tg].T
    assert relerr(got, ref) < 1e-5


@pytest.mark.parametrize("trunc,N", [(2, 333), (3, 1024), (3, 700), (2, 1300), (4, 1024)])
@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("wpt", [4, 8, 16])
def test_split_tail_matches_unsplit(ctx, gbi, trunc, N, precision, wpt):
    """The streaming form with the last, partly filled wave's targets split over several
    blocks (the default) sums the same pairs as without the split; three launches in a
    row (the arrival counters must be back at zero after each)."""
    s = workloads.small_cloud(N, 40 + N, phi=0.05)
    R = dev(s["R"])
    d = tensors.ModeBasis(trunc).d
    h = d - 6
    x = dev(np.random.default_rng(N + wpt).normal(size=(h, N)))
    ctx.set_wpt(wpt)
    ctx.set_split_tail(0)
    y_ref = torch.zeros((h, N), dtype=torch.float64, device="cuda")
    ctx.apply(N, trunc, 1.0, 2, 2, precision, R, x, y_ref, 1.0, 0.0, True)
    ctx.set_split_tail(1)
    for _ in range(3):
        y = torch.full((h, N), 7.0, dtype=torch.float64, device="cuda")
        ctx.apply(N, trunc, 1.0, 2, 2, precision, R, x, y, 1.0, 0.0, True)
        torch.cuda.synchronize()
        assert relerr(y.cpu().numpy(), y_ref.cpu().numpy()) < (2e-6 if precision == 1 else 1e-12)
    ctx.set_wpt(0)


@pytest.mark.parametrize("precision,tol", [(1, 1e-5), (2, 1e-11)])
def test_split_tail_full_size_sampled_rows(ctx, gbi, precision, tol):
    """N = 1024 at l <= 3 with 4 warps per target (608 resident blocks: the last 416 targets
    split), against the oracle's dense pair blocks for sampled targets of both waves."""
    c = workloads.config2()
    R = c["R"]
    N, trunc = len(R), 3
    d = tensors.ModeBasis(trunc).d
    h = d - 6
    x = np.random.default_rng(6).normal(size=(h, N))
    ctx.set_wpt(4)
    y = torch.zeros((h, N), dtype=torch.float64, device="cuda")
    ctx.apply(N, trunc, c["a"], 2, 2, precision, dev(R), dev(x), y, 1.0, 0.0, False)
    torch.cuda.synchronize()
    ctx.set_wpt(0)
    tg = np.array([0, 300, 607, 608, 609, 900, 1023])
    xf = np.zeros((N, d))
    xf[:, 6:] = x.T
    ref = galerkin.apply_offdiag(R, xf, c["a"], trunc, rows=slice(6, d), targets=tg)
    got = y.cpu().numpy()[:, tg].T
    assert relerr(got, ref) < tol
