"""The mixed-precision solve replayed as one CUDA graph, every decision on the device
(refinement sweeps, GMRES restarts and Arnoldi steps as nested conditional nodes).

The graph launches the kernels of the host-driven sequence in the same order, so a
replayed solve must give that sequence's V, Omega, Q^H bit for bit and the same
counters; the host-driven sequence itself is checked against the FP64 oracle in
test_gpu_parity.py.  Cases: single and batched suspensions, every mixed precision,
new input values under the same key, a key change, the iteration cap, the overlap
guard.
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


def inputs(sizes, trunc, seed, scale=1.0):
    Rs, ps, offs = [], [], [0]
    for k, n in enumerate(sizes):
        c = workloads.small_cloud(n, seed + k, phi=0.05)
        Rs.append(c["R"] + 200.0 * k)
        ps.append(c["p"])
        offs.append(offs[-1] + n)
    R, p = np.concatenate(Rs), np.concatenate(ps)
    prm_o = dict(a=1.0, eta=workloads.ETA_DEFAULT, k=0.01, vs=0.1 * scale, s0=0.05, d0=0.02)
    inp = dynamics.trap_inputs(R, p, prm_o, trunc)
    inp["Te"] = np.random.default_rng(seed).normal(size=(len(R), 3)) * 0.01
    return R, {k: dev(v) for k, v in inp.items()}, offs


INFO = ("iters", "refinements", "matvecs_f32", "matvecs_f64", "pair_interactions", "rel_residual",
        "min_separation")


def run(gbi, ctx, prm, R, t, offs, batched, **kw):
    if batched:
        out = ctx.batch_solve(prm, offs, dev(R), t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"], **kw)
    else:
        out = ctx.solve(prm, dev(R), t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"], **kw)
    torch.cuda.current_stream().synchronize()
    V, O, Q, info, st = out
    return V.clone(), O.clone(), Q.clone(), {k: getattr(info, k) for k in INFO}, st


def same(a, b):
    for x, y in zip(a[:3], b[:3]):
        assert torch.equal(x, y)
    assert a[3] == b[3]
    assert a[4] == b[4]


@pytest.mark.parametrize("batched,sizes,trunc", [(False, [48], 3), (False, [40], 2), (True, [30, 64, 9], 2),
                                                 (True, [20, 33], 3)])
@pytest.mark.parametrize("precision", [1, 2, 3])
def test_replay_matches_host_sequence(gbi, batched, sizes, trunc, precision):
    R, t, offs = inputs(sizes, trunc, seed=40 + trunc)
    prm = gbi.params(a=1.0, eta=workloads.ETA_DEFAULT, trunc=trunc, precision=precision, rtol=1e-10)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gbi.Context(0, stream=stream)
        first = run(gbi, ctx, prm, R, t, offs, batched)           # host-driven
        assert ctx.solve_graph_replays() == 0
        for k in range(2):                                        # built, then replayed
            same(run(gbi, ctx, prm, R, t, offs, batched), first)
            assert ctx.solve_graph_replays() == k + 1
        assert first[3]["rel_residual"] <= 1e-10 and first[3]["refinements"] >= 1
        # new values in the same buffers: the replay follows them
        R2, t2, _ = inputs(sizes, trunc, seed=40 + trunc, scale=1.7)
        for k in t:
            t[k].copy_(t2[k])
        rep = run(gbi, ctx, prm, R, t, offs, batched)
        assert ctx.solve_graph_replays() == 3
        ctx.close()
        fresh = gbi.Context(0, stream=stream)
        same(rep, run(gbi, fresh, prm, R, t, offs, batched))
        assert fresh.solve_graph_replays() == 0
        fresh.close()


@pytest.mark.parametrize("precision", [1, 3])
def test_replay_matches_host_sequence_many_systems(gbi, precision):
    """64 systems or more take the separate dot-product and Givens kernels."""
    sizes = [int(n) for n in np.random.default_rng(5).integers(2, 14, size=70)]
    R, t, offs = inputs(sizes, 2, seed=60)
    prm = gbi.params(a=1.0, eta=workloads.ETA_DEFAULT, trunc=2, precision=precision, rtol=1e-10)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gbi.Context(0, stream=stream)
        first = run(gbi, ctx, prm, R, t, offs, True)
        for k in range(2):
            same(run(gbi, ctx, prm, R, t, offs, True), first)
            assert ctx.solve_graph_replays() == k + 1
        assert first[3]["rel_residual"] <= 1e-10
        ctx.close()


@pytest.mark.parametrize("restart", [2, 64])
def test_replay_with_short_and_long_restarts(gbi, restart):
    """Restart 2: many GMRES cycles per inner solve (the restart loop of the graph);
    restart 64: Krylov dimensions past the triangular solve's shared-memory stage."""
    R, t, offs = inputs([96], 3, seed=70)
    # an inner tolerance below the FP32 floor makes every cycle run its full length
    prm = gbi.params(a=1.0, eta=workloads.ETA_DEFAULT, trunc=3, precision=2, rtol=1e-10, restart=restart,
                     max_iter=4000, max_refine=30, inner_rtol=1e-5 if restart == 2 else 1e-12)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gbi.Context(0, stream=stream)
        first = run(gbi, ctx, prm, R, t, offs, False)
        for k in range(2):
            same(run(gbi, ctx, prm, R, t, offs, False), first)
        assert ctx.solve_graph_replays() == 2
        assert first[3]["rel_residual"] <= 1e-10
        ctx.close()


def test_key_change_and_launch_count(gbi):
    R, t, offs = inputs([48], 3, seed=7)
    prm = gbi.params(a=1.0, eta=workloads.ETA_DEFAULT, trunc=3, precision=3, rtol=1e-10)
    prm2 = gbi.params(a=1.0, eta=workloads.ETA_DEFAULT, trunc=3, precision=3, rtol=1e-8)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gbi.Context(0, stream=stream)
        l0 = ctx.kernel_launches()
        a = run(gbi, ctx, prm, R, t, offs, False)
        host_launches = ctx.kernel_launches() - l0
        same(run(gbi, ctx, prm, R, t, offs, False), a)
        l1 = ctx.kernel_launches()
        same(run(gbi, ctx, prm, R, t, offs, False), a)
        # a replay counts the kernels its graph ran: about the host-driven sequence's
        # (the per-cycle graph and the one-off set-up launches differ by a few)
        assert abs((ctx.kernel_launches() - l1) - host_launches) <= 0.25 * host_launches
        assert ctx.solve_graph_replays() == 2
        b = run(gbi, ctx, prm2, R, t, offs, False)                # new key: host-driven again
        assert ctx.solve_graph_replays() == 2
        assert b[3]["rel_residual"] <= 1e-8
        same(run(gbi, ctx, prm2, R, t, offs, False), b)
        assert ctx.solve_graph_replays() == 3
        same(run(gbi, ctx, prm, R, t, offs, False), a)           # and back
        ctx.close()


def test_iteration_cap_and_refinement_cap(gbi):
    R, t, offs = inputs([48], 3, seed=9)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for kw in (dict(max_iter=5), dict(max_refine=1), dict(max_iter=12, max_refine=2)):
            prm = gbi.params(a=1.0, eta=workloads.ETA_DEFAULT, trunc=3, precision=2, rtol=1e-10, **kw)
            ctx = gbi.Context(0, stream=stream)
            res = [run(gbi, ctx, prm, R, t, offs, False, allow_not_converged=True) for _ in range(3)]
            assert ctx.solve_graph_replays() == 2
            same(res[1], res[0])
            same(res[2], res[0])
            assert res[0][4] == gbi.GBI_ERR_NOT_CONVERGED
            if "max_iter" in kw:
                assert res[0][3]["iters"] <= kw["max_iter"]
            ctx.close()


def test_overlap_guard_in_the_graph(gbi):
    R, t, offs = inputs([20], 2, seed=11)
    R = R.copy()
    R[1] = R[0] + np.array([1.5, 0.0, 0.0])    # centres 1.5 a apart
    prm = gbi.params(a=1.0, eta=workloads.ETA_DEFAULT, trunc=2, precision=3, rtol=1e-10, min_sep=2.0)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gbi.Context(0, stream=stream)
        for _ in range(3):
            with pytest.raises(RuntimeError, match="overlap"):
                run(gbi, ctx, prm, R, t, offs, False)
        assert ctx.solve_graph_replays() == 2
        ctx.close()


def _trap_case(gbi, precision, max_iter=1000):
    c = workloads.config1()
    prm = gbi.params(a=c["a"], eta=c["eta"], trunc=3, precision=precision, rtol=1e-10, max_iter=max_iter)
    return c, prm


@pytest.mark.parametrize("precision", [2, 3])
def test_trap_steps_replayed_with_their_inputs_and_update(gbi, precision):
    """A trap step replays its inputs, solve and Euler update as one graph: every replayed
    step equals a host-driven step taken from the same state on a fresh context."""
    c, prm = _trap_case(gbi, precision)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gbi.Context(0, stream=stream)
        R = dev(c["R"])
        p = dev(c["p"])
        for k in range(4):
            R0, p0 = R.clone(), p.clone()
            info = ctx.trap_step(prm, R, p, 0.05, c["k"], c["vs"], c["s0"], c["d0"], False, 1)
            stream.synchronize()
            assert info.rel_residual <= 1e-10
            ref = gbi.Context(0, stream=stream)
            R1, p1 = R0.clone(), p0.clone()
            ref.trap_step(prm, R1, p1, 0.05, c["k"], c["vs"], c["s0"], c["d0"], False, 1)
            stream.synchronize()
            assert ref.solve_graph_replays() == 0
            assert torch.equal(R1, R) and torch.equal(p1, p), k
            ref.close()
        # steps 1 and 2 repeat step 0's key only in sizes: R moved, but its buffer did not
        assert ctx.solve_graph_replays() >= 2
        ctx.close()


def test_failed_trap_step_leaves_the_state_in_the_graph(gbi):
    c, prm = _trap_case(gbi, 3, max_iter=3)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = gbi.Context(0, stream=stream)
        R = dev(c["R"])
        p = dev(c["p"])
        R0, p0 = R.clone(), p.clone()
        for _ in range(3):
            with pytest.raises(gbi.GbiError):
                ctx.trap_step(prm, R, p, 0.05, c["k"], c["vs"], c["s0"], c["d0"], False, 1)
            stream.synchronize()
            assert torch.equal(R, R0) and torch.equal(p, p0)
        assert ctx.solve_graph_replays() == 2
        ctx.close()
