"""gbi_solve_static: the solve for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc while they run (a framework that owns every
allocation, a real-time loop, a pre-planned memory budget).  gbi_solve_static takes
its whole workspace from one static device array inside the library.  These tests
call it through the C ABI and compare it with gbi_solve, which allocates its
workspace in a context, on two calls in a row with different inputs (so stale
contents of the shared array would show) -- in every precision, with and without a
warm start, at the largest sizes the array admits and on a caller's stream -- check that
no device memory is taken by a call, and that sizes beyond the stated limits are
refused before any work.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle import dynamics

pytestmark = pytest.mark.gpu

TOL = 1e-12     # same arithmetic on the same inputs: agreement to FP64 rounding


def _inputs(N, seed, trunc):
    s = workloads.small_cloud(N, seed)
    prm_o = dict(a=s["a"], eta=s["eta"], k=s["k"], vs=s["vs"], s0=s["s0"], d0=0.02)
    inp = dynamics.trap_inputs(s["R"], s["p"], prm_o, trunc)
    inp["Te"] = np.random.default_rng(seed).normal(size=(N, 3)) * 0.01
    inp["R"] = s["R"]
    t = {k: torch.tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda") for k, v in inp.items()}
    return s, t


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.fixture(scope="module")
def gbi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_0278_gb300 as g
    g.lib()
    return g


def _compare_twice(gbi, trunc, N, precision, warm_start, stream=None):
    """Two calls in a row with different inputs: the static entry point against the context
    solve (same kernels, same order: FP64 rounding agreement).  With warm_start the second
    call starts from the first call's solution."""
    # the context solve runs host-driven on the default stream (a context on a caller's
    # stream would replay a CUDA graph with another kernel sequence); the static call
    # runs on `stream`
    ctx = gbi.Context(0)
    Q_init = torch.zeros((N, gbi.h(trunc)), dtype=torch.float64, device="cuda")
    try:
        for call, seed in enumerate((41, 42)):
            s, t = _inputs(N, seed, trunc)
            prm = gbi.params(a=s["a"], eta=s["eta"], trunc=trunc, precision=precision, rtol=1e-10, restart=32)
            Qc = Q_init.clone()
            V0, O0, Q0, i0, st0 = ctx.solve(prm, t["R"], t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"], QH=Qc,
                                            warm_start=warm_start)
            V = torch.full_like(V0, float("nan"))
            O = torch.full_like(O0, float("nan"))
            Q = Q_init.clone() if warm_start else torch.full_like(Q0, float("nan"))
            info, st = gbi.solve_static(prm, t["R"], t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"], V, O, Q,
                                        warm_start=warm_start, stream=stream)
            torch.cuda.synchronize()
            assert st == gbi.GBI_OK and st0 == gbi.GBI_OK, call
            assert info.rel_residual <= 1e-10
            assert _rel(V, V0) < TOL and _rel(O, O0) < TOL and _rel(Q, Q0) < TOL, call
            assert info.iters == i0.iters and info.pair_interactions == i0.pair_interactions
            Q_init = Q0.clone()   # a warm start from the previous call's solution
    finally:
        ctx.close()


@pytest.mark.parametrize("trunc,N", [(2, 300), (3, 200)])
def test_static_solve_matches_context_solve_twice(gbi, trunc, N):
    _compare_twice(gbi, trunc, N, 1, False)


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
@pytest.mark.parametrize("warm_start", [False, True])
@pytest.mark.parametrize("trunc,N", [(2, 1024), (3, 327)])
def test_static_solve_every_precision_at_the_size_limits(gbi, precision, warm_start, trunc, N):
    """The largest sizes the static array admits (N = 1024 at l <= 2; N h = 8175 at l <= 3),
    every arithmetic (FP64, FP32 with FP64 or double-float refinement, FP32 right-hand
    side) and a warm start: every workspace slot is exercised at its bound."""
    _compare_twice(gbi, trunc, N, precision, warm_start)


def test_static_solve_on_a_caller_stream_allocates_nothing(gbi):
    """On a caller's stream: results as on the default stream, and no device memory is
    taken between a second and a third call (cudaMemGetInfo free bytes unchanged)."""
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        _compare_twice(gbi, 3, 200, 3, False, stream=stream)
        s, t = _inputs(200, 43, 3)
        prm = gbi.params(a=s["a"], eta=s["eta"], trunc=3, precision=3, rtol=1e-10, restart=32)
        V = torch.zeros((200, 3), dtype=torch.float64, device="cuda")
        O = torch.zeros_like(V)
        Q = torch.zeros((200, 25), dtype=torch.float64, device="cuda")
        gbi.solve_static(prm, t["R"], t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"], V, O, Q, stream=stream)
        stream.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        info, st = gbi.solve_static(prm, t["R"], t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"], V, O, Q,
                                    stream=stream)
        stream.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    assert st == gbi.GBI_OK and info.rel_residual <= 1e-10
    assert free1 == free0


def test_static_solve_refuses_sizes_beyond_limits(gbi):
    z = lambda *shape: torch.zeros(shape, dtype=torch.float64, device="cuda")
    N = 1025                                   # above the 1024-sphere limit
    prm = gbi.params(a=1.0, eta=1.0, trunc=2)
    with pytest.raises(gbi.GbiError) as e:
        gbi.solve_static(prm, z(N, 3), z(N, 3), z(N, 3), z(N, 8), z(N, 3), z(N, 3), z(N, 3), z(N, 3), z(N, 8))
    assert e.value.status == gbi.GBI_ERR_ARG
    N = 400                                    # 400 x 25 > 8192 higher components
    prm = gbi.params(a=1.0, eta=1.0, trunc=3)
    with pytest.raises(gbi.GbiError):
        gbi.solve_static(prm, z(N, 3), z(N, 3), z(N, 3), z(N, 25), z(N, 3), z(N, 3), z(N, 3), z(N, 3), z(N, 25))
    prm = gbi.params(a=1.0, eta=1.0, trunc=2, restart=33)
    with pytest.raises(gbi.GbiError):
        gbi.solve_static(prm, z(8, 3), z(8, 3), z(8, 3), z(8, 8), z(8, 3), z(8, 3), z(8, 3), z(8, 3), z(8, 8))
