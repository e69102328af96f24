"""Squirmers (Sec. V): their active modes on the GPU and two squirmers in a harmonic trap.

The GPU writes the squirmer modes in closed form (gbi_squirmer_inputs); the oracle
projects the printed Lighthill-Blake slip onto its own mode basis (pinned in
test_oracle_pins.py).  Two squirmers on the trap sphere R* = 12.56 a (Sec. V, two-particle
discussion): diametrically opposite (theta0 = 180 degrees) they do not rotate; at any
other angle they do; a few re-solved steps follow the oracle's trajectory.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle import dynamics, galerkin

pytestmark = pytest.mark.gpu

B1, B2 = 0.15, -1.0 / 12.0          # V^a = 0.1 p, V^(2s) = 0.05 (pp - I/3)
RSTAR = 12.56
ETA = workloads.ETA_DEFAULT
K_TRAP = 6 * math.pi * ETA * (2 * B1 / 3) / RSTAR     # R* = 6 pi eta v_s a / k


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


def pair_on_trap_sphere(theta0_deg):
    """Particle 1 at the north pole, particle 2 at theta0 from it (in the x-z plane),
    both on the sphere of radius R* and pointing outwards."""
    t = math.radians(theta0_deg)
    u = np.array([[0.0, 0.0, 1.0], [math.sin(t), 0.0, math.cos(t)]])
    return RSTAR * u, u.copy()


@pytest.mark.parametrize("trunc", [2, 3, 4])
def test_squirmer_inputs_match_the_slip_projection(ctx, gbi, trunc):
    rng = np.random.default_rng(trunc)
    p = rng.normal(size=(7, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    R = rng.normal(size=(7, 3)) * 5
    got = ctx.squirmer_inputs(7, trunc, K_TRAP, B1, B2, dev(R), dev(p))
    torch.cuda.synchronize()
    for n in range(7):
        Va, Oa, VH = dynamics.squirmer_modes(p[n], B1, B2, trunc)
        assert np.abs(got["Va"][n].cpu().numpy() - Va).max() < 1e-14
        assert np.abs(got["VH"][n].cpu().numpy() - VH).max() < 1e-13
    assert np.abs(got["Oa"].cpu().numpy()).max() == 0.0
    np.testing.assert_allclose(got["Fe"].cpu().numpy(), -K_TRAP * R, rtol=1e-15)


@pytest.mark.parametrize("superposition,precision", [(True, 1), (False, 0)])
def test_opposite_pair_is_frozen(ctx, gbi, superposition, precision):
    """theta0 = 180 degrees: the configuration is symmetric about the line through both
    spheres, so neither rotates (p stays fixed) and both stay on that line."""
    R, p = pair_on_trap_sphere(180.0)
    prm = gbi.params(a=1.0, eta=ETA, trunc=2, precision=precision, rtol=1e-10)
    Rd, pd = dev(R), dev(p)
    ctx.squirmer_step(prm, Rd, pd, 0.5, K_TRAP, B1, B2, superposition, 200)
    torch.cuda.synchronize()
    Rn, pn = Rd.cpu().numpy(), pd.cpu().numpy()
    assert np.abs(pn - p).max() < 1e-12
    assert np.abs(Rn[:, :2]).max() < 1e-9 * RSTAR


def test_other_angles_rotate(ctx, gbi):
    R, p = pair_on_trap_sphere(115.0)
    prm = gbi.params(a=1.0, eta=ETA, trunc=2, precision=1)
    Rd, pd = dev(R), dev(p)
    ctx.squirmer_step(prm, Rd, pd, 0.5, K_TRAP, B1, B2, True, 200)
    torch.cuda.synchronize()
    assert np.abs(pd.cpu().numpy() - p).max() > 1e-4


def test_squirmer_steps_match_oracle(ctx, gbi):
    """Three forward-Euler steps of the full l <= 3 solve (FP64) for two squirmers at
    theta0 = 115 degrees, against the oracle's solve with its projected squirmer modes."""
    trunc, dt, n = 3, 0.5, 3
    R, p = pair_on_trap_sphere(115.0)
    Rr, pr = R.copy(), p.copy()
    z = np.zeros((2, 3))
    for _ in range(n):
        modes = [dynamics.squirmer_modes(pr[i], B1, B2, trunc) for i in range(2)]
        Va = np.array([m[0] for m in modes])
        VH = np.array([m[2] for m in modes])
        V, Om, _ = galerkin.solve(Rr, Va, z, VH, -K_TRAP * Rr, z, 1.0, ETA, trunc)
        Rr, pr = dynamics.euler(Rr, pr, V, Om, dt)
    prm = gbi.params(a=1.0, eta=ETA, trunc=trunc, precision=0, rtol=1e-12)
    Rd, pd = dev(R), dev(p)
    ctx.squirmer_step(prm, Rd, pd, dt, K_TRAP, B1, B2, False, n)
    torch.cuda.synchronize()
    assert np.abs(Rd.cpu().numpy() - Rr).max() < 1e-11 * RSTAR
    assert np.abs(pd.cpu().numpy() - pr).max() < 1e-10
