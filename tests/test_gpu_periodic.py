"""Point-force superposition in a periodic cube (gbi_periodic_superpose) against the
oracle's direct Ewald lattice sums (oracle/periodic.py, pinned by splitting-parameter
independence, Hasimoto's self mobility and a supercell of a simple cubic array).

The GPU chooses its own split (cells per side, splitting parameter, wave-vector cut-off)
and its wave-space form (direct sums or the particle mesh); results must not depend on
them: every pair (minimum image) and cell lists of 3..6 cells per side give the same
velocities.  FP64 to 1e-11 of the largest velocity, FP32 to 1e-5.  The mesh converges to
the direct sum as the mesh is refined (spline order 8: error ~ K^-10), FP64 to 1e-7 at
K = 7.6 xi L; FP32 meshes to 1e-5.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import periodic

pytestmark = pytest.mark.gpu

A, ETA = 1.0, 0.7


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


def box(N, L, seed, dmin=2.2):
    """N centres in the cube [0, L)^3 (shifted by whole cells at random, as positions
    outside the cell are allowed), at least dmin apart by the minimum image."""
    rng = np.random.default_rng(seed)
    R = np.zeros((N, 3))
    n = 0
    while n < N:
        x = rng.uniform(0, L, size=3)
        d = (x - R[:n]) - L * np.rint((x - R[:n]) / L)
        if n == 0 or (d * d).sum(1).min() >= dmin * dmin:
            R[n] = x
            n += 1
    R = R + L * rng.integers(-2, 3, size=(N, 3))
    F = rng.normal(size=(N, 3)) * 0.1
    Va = rng.normal(size=(N, 3)) * 0.01
    return R, F, Va


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-5)])
def test_periodic_matches_oracle(ctx, gbi, precision, tol):
    L = 12.0
    R, F, Va = box(40, L, 1)
    V_o = periodic.periodic_superpose(R, Va, F, A, ETA, L, nmax=3, mmax=12)
    prm = gbi.params(a=A, eta=ETA, trunc=2, precision=precision)
    V, plan = ctx.periodic_superpose(prm, L, dev(R), dev(Va), dev(F))
    torch.cuda.synchronize()
    scale = np.abs(V_o - Va).max()
    assert np.abs(V.cpu().numpy() - V_o).max() <= tol * scale, plan


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-5)])
def test_split_does_not_matter(ctx, gbi, precision, tol):
    """Every pair by the minimum image and cell lists of 3..6 cells per side."""
    L = 40.0
    R, F, Va = box(1500, L, 2)
    prm = gbi.params(a=A, eta=ETA, trunc=2, precision=precision)
    V0, p0 = ctx.periodic_superpose(prm, L, dev(R), dev(Va), dev(F), cells=-1)
    assert p0["cells_per_side"] == 0 and p0["mesh"] == 0
    ref = V0.cpu().numpy()
    scale = np.abs(ref - Va).max()
    for M in (3, 4, 6):
        V, plan = ctx.periodic_superpose(prm, L, dev(R), dev(Va), dev(F), cells=M, mesh=-1)
        torch.cuda.synchronize()
        assert plan["cells_per_side"] == M and plan["mesh"] == 0
        assert np.abs(V.cpu().numpy() - ref).max() <= tol * scale, (M, plan)
    # and the oracle for a few spheres
    tg = [0, 777, 1499]
    V_o = periodic.periodic_superpose(R, Va, F, A, ETA, L, targets=tg, nmax=2, mmax=12)
    assert np.abs(ref[tg] - V_o).max() <= max(tol, 1e-11) * scale


def test_simple_cubic_array_moves_with_hasimotos_correction(ctx, gbi):
    """A 4 x 4 x 4 simple cubic array of equal forces in a box of 4 cells: every sphere moves
    at F/(6 pi eta a) (1 - 2.837297 a / L), L the lattice spacing."""
    L = 5.0
    g = np.arange(4) * L
    R = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 0.37
    F = np.tile([0.3, -0.2, 0.1], (64, 1))
    z = np.zeros_like(F)
    prm = gbi.params(a=A, eta=ETA, trunc=2, precision=0)
    for cells in (0, 3, -1):
        V, plan = ctx.periodic_superpose(prm, 4 * L, dev(R), dev(z), dev(F), cells=cells)
        torch.cuda.synchronize()
        want = F[0] / (6 * math.pi * ETA * A) * (1 - 2.837297 * A / L)
        np.testing.assert_allclose(V.cpu().numpy(), np.tile(want, (64, 1)), rtol=1e-6)
        V1 = periodic.periodic_superpose(R[:1], z[:1], F[:1], A, ETA, L, nmax=3, mmax=12)
        np.testing.assert_allclose(V.cpu().numpy(), np.tile(V1, (64, 1)), rtol=1e-11)


def test_mesh_converges_to_the_direct_sum_fp64(ctx, gbi):
    """FP64 meshes of 32, 64 and 128 points per side (3 cells per side, xi L = 16.8): the
    error against the direct sum falls by ~2^10 per doubling and reaches 1e-7."""
    L = 40.0
    R, F, Va = box(1500, L, 3)
    prm = gbi.params(a=A, eta=ETA, trunc=2, precision=0)
    V0, _ = ctx.periodic_superpose(prm, L, dev(R), dev(Va), dev(F), cells=3, mesh=-1)
    ref = V0.cpu().numpy()
    scale = np.abs(ref - Va).max()
    errs = []
    for K in (32, 64, 128):
        V, plan = ctx.periodic_superpose(prm, L, dev(R), dev(Va), dev(F), cells=3, mesh=K)
        torch.cuda.synchronize()
        assert plan["mesh"] == K and plan["cells_per_side"] == 3 and plan["n_wave"] == K ** 3
        errs.append(np.abs(V.cpu().numpy() - ref).max() / scale)
    assert errs[2] < 1e-7, errs
    assert errs[1] < errs[0] / 100 and errs[2] < errs[1] / 100, errs


@pytest.mark.parametrize("cells,K", [(3, 64), (4, 128), (6, 128)])
def test_mesh_fp32_matches_oracle(ctx, gbi, cells, K):
    """FP32 meshes against the FP64 direct sum (every sphere) and the oracle (sampled)."""
    L = 40.0
    R, F, Va = box(1500, L, 4)
    prm64 = gbi.params(a=A, eta=ETA, trunc=2, precision=0)
    V0, _ = ctx.periodic_superpose(prm64, L, dev(R), dev(Va), dev(F), cells=-1)
    ref = V0.cpu().numpy()
    scale = np.abs(ref - Va).max()
    prm = gbi.params(a=A, eta=ETA, trunc=2, precision=1)
    V, plan = ctx.periodic_superpose(prm, L, dev(R), dev(Va), dev(F), cells=cells, mesh=K)
    torch.cuda.synchronize()
    assert plan["mesh"] == K and plan["cells_per_side"] == cells
    Vg = V.cpu().numpy()
    assert np.abs(Vg - ref).max() <= 1e-5 * scale, plan
    tg = [5, 1234]
    V_o = periodic.periodic_superpose(R, Va, F, A, ETA, L, targets=tg, nmax=2, mmax=12)
    assert np.abs(Vg[tg] - V_o).max() <= 1e-5 * scale


def test_mesh_simple_cubic_array(ctx, gbi):
    """Hasimoto's correction through the mesh (FP32 and FP64)."""
    L = 5.0
    g = np.arange(4) * L
    R = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 0.37
    F = np.tile([0.3, -0.2, 0.1], (64, 1))
    z = np.zeros_like(F)
    want = F[0] / (6 * math.pi * ETA * A) * (1 - 2.837297 * A / L)
    for precision, K, tol in ((0, 128, 1e-6), (1, 64, 1e-5)):
        prm = gbi.params(a=A, eta=ETA, trunc=2, precision=precision)
        V, plan = ctx.periodic_superpose(prm, 4 * L, dev(R), dev(z), dev(F), cells=3, mesh=K)
        torch.cuda.synchronize()
        assert plan["mesh"] == K
        np.testing.assert_allclose(V.cpu().numpy(), np.tile(want, (64, 1)), rtol=tol, atol=tol * np.abs(want).max())


def test_mesh_chosen_at_large_n(ctx, gbi):
    """N = 2 10^4 at volume fraction 0.1 in FP32: the work estimate takes the mesh; every
    sphere within 1e-5 of the every-pair sum and sampled spheres of the oracle."""
    N = 20000
    L = (N * 4.0 * math.pi / 3.0 / 0.1) ** (1.0 / 3.0)
    rng = np.random.default_rng(21)
    R = rng.uniform(0.0, L, size=(N, 3))
    F = rng.normal(size=(N, 3)) * 0.1
    Va = np.zeros_like(R)
    prm = gbi.params(a=A, eta=ETA, trunc=2, precision=1)
    V, plan = ctx.periodic_superpose(prm, L, dev(R), dev(Va), dev(F))
    V0, p0 = ctx.periodic_superpose(prm, L, dev(R), dev(Va), dev(F), cells=-1, mesh=-1)
    torch.cuda.synchronize()
    assert plan["mesh"] >= 16 and plan["cells_per_side"] >= 3, plan
    ref = V0.cpu().numpy()
    scale = np.abs(ref).max()
    Vg = V.cpu().numpy()
    assert np.abs(Vg - ref).max() <= 1e-5 * scale, plan
    tg = [17, 19999]
    V_o = periodic.periodic_superpose(R, Va, F, A, ETA, L, targets=tg, nmax=2, mmax=14)
    assert np.abs(Vg[tg] - V_o).max() <= 1e-5 * scale


def test_mesh_argument_checks(ctx, gbi):
    R, F, Va = box(10, 12.0, 5)
    prm = gbi.params(a=A, eta=ETA, trunc=2, precision=1)
    for K in (8, 24, 1024):
        with pytest.raises(RuntimeError):
            ctx.periodic_superpose(prm, 12.0, dev(R), dev(Va), dev(F), cells=3, mesh=K)


def test_mesh_bench_workload_sampled(ctx, gbi):
    """The periodic bench workload (N = 10^5 at volume fraction 0.1, FP32): the chosen plan
    (particle mesh) against the every-pair sum on every sphere and the oracle's lattice sums
    for a sampled sphere."""
    N = 100000
    L = (N * 4.0 * math.pi / 3.0 / 0.1) ** (1.0 / 3.0)
    rng = np.random.default_rng(12345 + N)
    R = rng.uniform(0.0, L, size=(N, 3))
    F = rng.normal(size=(N, 3)) * 0.1
    Va = np.zeros_like(R)
    prm = gbi.params(a=A, eta=ETA, trunc=2, precision=1)
    V, plan = ctx.periodic_superpose(prm, L, dev(R), dev(Va), dev(F))
    torch.cuda.synchronize()
    assert plan["mesh"] > 0, plan
    V0, _ = ctx.periodic_superpose(prm, L, dev(R), dev(Va), dev(F), cells=-1, mesh=-1)
    torch.cuda.synchronize()
    ref = V0.cpu().numpy()
    scale = np.abs(ref).max()
    Vg = V.cpu().numpy()
    assert np.abs(Vg - ref).max() <= 1e-5 * scale, plan
    tg = [31337]
    V_o = periodic.periodic_superpose(R, Va, F, A, ETA, L, targets=tg, nmax=1, mmax=10)
    assert np.abs(Vg[tg] - V_o).max() <= 1e-5 * scale
