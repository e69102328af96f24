"""Trap dynamics on the GPU (Sec. V, Eq. trap_eom; Sec. II kinematics) against the oracle.

Two workloads, run through gbi_trap_step as the benchmark runs them:
* N = 64 active spheres, l <= 2, every step a full FP64 Galerkin solve to 1e-10, 100
  forward-Euler steps of dt = 0.1.  At steps 0, 50 and 100 the velocities the GPU
  computes on its own state are compared with the oracle's dense LU solve of that
  state (1e-9 of the largest velocity), and the first steps of the trajectory with the
  oracle's own trajectory.
* N = 10^4 spheres of the Gaussian trap cloud, superposition in FP32, dt = 0.05.  After
  25 and 50 steps the velocities on the GPU's state are compared with the oracle's
  superposition sum for sampled spheres (1e-5).  A chaotic many-step trajectory is not
  compared point by point (rounding differences grow), only per-step velocities.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle import dynamics, galerkin

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gbi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_0278_gb300 as g
    g.lib()
    return g


@pytest.fixture(scope="module")
def ctx(gbi):
    c = gbi.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel_rows(x, ref):
    """max_n |x_n - ref_n| / max_n |ref_n| over per-sphere 3-vectors."""
    return np.linalg.norm(x - ref, axis=1).max() / np.linalg.norm(ref, axis=1).max()


def _gpu_velocities(ctx, gbi, c, prm, R, p, superposition):
    N = len(R)
    Rd, pd = dev(R), dev(p)
    t = ctx.trap_inputs(N, c["trunc"], c["k"], c["vs"], c["s0"], c["d0"], Rd, pd)
    if superposition:
        V, Om = ctx.superpose(prm, Rd, t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"])
    else:
        V, Om, _, info, _ = ctx.solve(prm, Rd, t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"])
        assert info.rel_residual <= prm.rtol
    torch.cuda.synchronize()
    return V.cpu().numpy(), Om.cpu().numpy()


def test_fp64_solve_trajectory_n64(ctx, gbi):
    c = workloads.config1()
    N = len(c["R"])
    prm_o = dict(a=c["a"], eta=c["eta"], k=c["k"], vs=c["vs"], s0=c["s0"], d0=c["d0"])
    prm = gbi.params(a=c["a"], eta=c["eta"], trunc=c["trunc"], precision=0, rtol=c["rtol"])
    dt = c["dt"]
    # the first two steps against the oracle's own trajectory
    Rr, pr = dynamics.trajectory(c["R"], c["p"], prm_o, c["trunc"], dt, 2)
    Rd, pd = dev(c["R"]), dev(c["p"])
    ctx.trap_step(prm, Rd, pd, dt, c["k"], c["vs"], c["s0"], c["d0"], False, 2)
    torch.cuda.synchronize()
    assert np.abs(Rd.cpu().numpy() - Rr).max() < 1e-11 * np.abs(Rr).max()
    assert np.abs(pd.cpu().numpy() - pr).max() < 1e-10
    # steps 0, 50, 100: velocities on the GPU's own state
    Rd, pd = dev(c["R"]), dev(c["p"])
    done = 0
    for target in (0, 50, 100):
        if target > done:
            info = ctx.trap_step(prm, Rd, pd, dt, c["k"], c["vs"], c["s0"], c["d0"], False, target - done)
            torch.cuda.synchronize()
            assert info.rel_residual <= c["rtol"]
            done = target
        R, p = Rd.cpu().numpy(), pd.cpu().numpy()
        assert np.all(np.isfinite(R)) and np.allclose(np.linalg.norm(p, axis=1), 1.0, atol=1e-12)
        Vg, Og = _gpu_velocities(ctx, gbi, c, prm, R, p, False)
        Vr, Or = dynamics.velocities(R, p, prm_o, c["trunc"], False)
        assert rel_rows(Vg, Vr) < 1e-9, (target, rel_rows(Vg, Vr))
        assert rel_rows(Og, Or) < 1e-9, (target, rel_rows(Og, Or))
    assert done == c["steps"]


def test_fp32_superposition_trajectory_n10000(ctx, gbi):
    c = workloads.config3()
    N = len(c["R"])
    prm_o = dict(a=c["a"], eta=c["eta"], k=c["k"], vs=c["vs"], s0=c["s0"], d0=c["d0"])
    prm = gbi.params(a=c["a"], eta=c["eta"], trunc=2, precision=1)
    Rd, pd = dev(c["R"]), dev(c["p"])
    rng = np.random.default_rng(3)
    for chunk in (25, 25):
        ctx.trap_step(prm, Rd, pd, c["dt"], c["k"], c["vs"], c["s0"], c["d0"], True, chunk)
        torch.cuda.synchronize()
        R, p = Rd.cpu().numpy(), pd.cpu().numpy()
        assert np.all(np.isfinite(R))
        Vg, Og = _gpu_velocities(ctx, gbi, c, prm, R, p, True)
        tg = rng.choice(N, size=10, replace=False)
        inp = dynamics.trap_inputs(R, p, prm_o, 2)
        Vr, Or = galerkin.superpose(R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"], c["a"], c["eta"], 2,
                                    targets=tg)
        assert rel_rows(Vg[tg], Vr) < 1e-5
        assert rel_rows(Og[tg], Or) < 1e-5


@pytest.mark.parametrize("superposition,precision", [(True, 1), (False, 3), (False, 0)])
def test_batched_trap_steps_match_per_system_steps(ctx, gbi, superposition, precision):
    """gbi_batch_trap_step on three suspensions of uneven size (each with its own trap at
    its origin) against gbi_trap_step on each system alone: the same trajectories, to the
    solve tolerance (lock-step batched GMRES sums in another order)."""
    sizes = [17, 40, 9]
    cs = [workloads.small_cloud(n, 300 + i) for i, n in enumerate(sizes)]
    offs = [0]
    for n in sizes:
        offs.append(offs[-1] + n)
    R = np.concatenate([c["R"] for c in cs])
    p = np.concatenate([c["p"] for c in cs])
    c = cs[0]
    prm = gbi.params(a=c["a"], eta=c["eta"], trunc=2, precision=precision, rtol=1e-10)
    Rb, pb = dev(R), dev(p)
    ctx.batch_trap_step(prm, offs, Rb, pb, 0.1, c["k"], c["vs"], c["s0"], 0.02, superposition, 3)
    torch.cuda.synchronize()
    for q in range(len(sizes)):
        Rs, ps = dev(R[offs[q]:offs[q + 1]]), dev(p[offs[q]:offs[q + 1]])
        one = gbi.Context(0)
        one.trap_step(prm, Rs, ps, 0.1, c["k"], c["vs"], c["s0"], 0.02, superposition, 3)
        torch.cuda.synchronize()
        one.close()
        Rr, pr = Rs.cpu().numpy(), ps.cpu().numpy()
        tol = 1e-6 if precision in (1, 3) else 1e-11
        assert np.abs(Rb.cpu().numpy()[offs[q]:offs[q + 1]] - Rr).max() < tol * np.abs(Rr).max()
        assert np.abs(pb.cpu().numpy()[offs[q]:offs[q + 1]] - pr).max() < tol


def test_batched_trap_step_replays_one_graph_per_step(gbi):
    """On a non-default stream a repeated mixed-precision batched step is one CUDA graph:
    trap inputs, the batched solve and the update of every system."""
    sizes = [30, 64, 12]
    cs = [workloads.small_cloud(n, 310 + i) for i, n in enumerate(sizes)]
    offs = [0]
    for n in sizes:
        offs.append(offs[-1] + n)
    R = dev(np.concatenate([c["R"] for c in cs]))
    p = dev(np.concatenate([c["p"] for c in cs]))
    c = cs[0]
    prm = gbi.params(a=c["a"], eta=c["eta"], trunc=2, precision=3, rtol=1e-10)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bctx = gbi.Context(0, stream=stream)
        for _ in range(4):
            bctx.batch_trap_step(prm, offs, R, p, 0.05, c["k"], c["vs"], c["s0"], 0.0, False, 1)
        stream.synchronize()
        assert bctx.solve_graph_replays() >= 2
        bctx.close()
    assert np.all(np.isfinite(R.cpu().numpy()))
