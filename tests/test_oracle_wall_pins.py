"""Pins of the wall oracle (oracle/wall.py) against what the mathematics fixes.

* no slip: the flow of a point force, and of a force dipole (stresslet and rotlet),
  plus its images vanishes on the wall z = 0;
* reciprocity of the wall Green's function, G^B_ij(x, y) = G^B_ji(y, x);
* the images' own value at the source: the classical wall corrections of a point
  force's mobility, 1 - 9a/(16h) parallel and 1 - 9a/(8h) normal to the wall;
* a force dipole (pusher) near the wall: the wall-normal velocity
  -3p (1 - 3 sin^2 theta) / (64 pi eta h^2) and the rotation rate
  -3p sin theta cos theta / (64 pi eta h^3) of a sphere (Berke et al. 2008);
* the force-dipole conventions: the dipole tensor gives the unbounded stresslet and
  rotlet flows, and S = (20/3) pi eta a^2 V^(2s) is the far field of the unbounded
  superposition's active strain term;
* the images fade far from the wall, and the derivatives of the forward-mode
  arithmetic agree with central differences.
"""
import math

import numpy as np
import pytest

from oracle import galerkin, tensors, wall


def oseen_jets(x, y):
    xj = [wall.Jet.var(x[k], k) for k in range(3)]
    yj = [wall.Jet.var(y[k], 3 + k) for k in range(3)]
    r = [xj[k] - yj[k] for k in range(3)]
    ir = (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]).sqrt().inv()
    ir3 = ir * ir * ir
    return [[(ir if i == j else 0.0) + r[i] * r[j] * ir3 for j in range(3)] for i in range(3)]


def dipole_flow(G, D):
    """u_i = D_jk d/dy_k G_ij (times 8 pi eta)."""
    return np.array([sum(np.dot(D[j], G[i][j].g[3:]) for j in range(3)) for i in range(3)])


def random_source(rng):
    y = rng.normal(size=3) * 2
    y[2] = rng.uniform(0.5, 4.0)
    return y


def test_no_slip_on_the_wall():
    rng = np.random.default_rng(1)
    for _ in range(20):
        y = random_source(rng)
        x = rng.normal(size=3) * 3
        x[2] = 0.0
        GB = wall.blake(x, y)
        assert np.abs(GB).max() < 1e-13 * np.abs(np.eye(3) / np.linalg.norm(x - y)).max()
        # force dipole: direct + image flow
        D = rng.normal(size=(3, 3))
        u = dipole_flow(oseen_jets(x, y), D) + dipole_flow(wall.image_jets(x, y), D)
        assert np.abs(u).max() < 1e-12 * np.abs(D).max() / np.linalg.norm(x - y) ** 2


def test_reciprocity():
    rng = np.random.default_rng(2)
    for _ in range(20):
        x, y = random_source(rng), random_source(rng)
        np.testing.assert_allclose(wall.blake(x, y), wall.blake(y, x).T, atol=1e-14, rtol=1e-12)


@pytest.mark.parametrize("h", [1.5, 4.0, 20.0])
def test_point_force_mobility_near_the_wall(h):
    """Image part at the source: -(3/(4h)) parallel and -(3/(2h)) normal (times
    F / (8 pi eta)), i.e. mobilities (1 - 9a/(16h)) and (1 - 9a/(8h)) / (6 pi eta a)."""
    y = np.array([0.3, -0.7, h])
    W = np.array([[w.v for w in row] for row in wall.image_jets(y, y)])
    np.testing.assert_allclose(np.diag(W), [-0.75 / h, -0.75 / h, -1.5 / h], rtol=1e-13)
    assert np.abs(W - np.diag(np.diag(W))).max() < 1e-14 / h
    a, eta = 1.0, 0.7
    mob = 1.0 / (6 * np.pi * eta * a) + np.diag(W) / (8 * np.pi * eta)
    np.testing.assert_allclose(mob * 6 * np.pi * eta * a, [1 - 9 * a / (16 * h), 1 - 9 * a / (16 * h),
                                                             1 - 9 * a / (8 * h)], rtol=1e-13)


@pytest.mark.parametrize("theta", [0.0, 0.3, 0.7, 1.2, math.pi / 2])
def test_pusher_near_the_wall(theta):
    """A force dipole p e e (pusher for p > 0), e at angle theta to the wall, at height h:
    its image flow at its own centre moves it along z and turns e toward the wall plane."""
    h, p, eta = 3.0, 1.3, 0.7
    e = np.array([math.cos(theta), 0.0, math.sin(theta)])
    D = p * (np.outer(e, e) - np.eye(3) / 3)
    y = np.array([0.2, 0.1, h])
    u, curl = wall.image_velocity(y, y, np.zeros(3), D)
    u /= 8 * np.pi * eta
    Om = 0.5 * curl / (8 * np.pi * eta)
    uz = -3 * p * (1 - 3 * math.sin(theta) ** 2) / (64 * np.pi * eta * h ** 2)
    assert u[2] == pytest.approx(uz, rel=1e-12, abs=1e-15)
    assert abs(u[1]) < 1e-15
    edot = np.cross(Om, e)
    thdot = edot[2] / math.cos(theta) if abs(math.cos(theta)) > 0.5 else -edot[0] / math.sin(theta)
    want = -3 * p * math.sin(theta) * math.cos(theta) / (64 * np.pi * eta * h ** 3)
    assert thdot == pytest.approx(want, rel=1e-12, abs=1e-15)


def test_force_dipole_conventions():
    """D_jk d/dy_k G_ij: the stresslet S gives 3 r (r.S.r) / r^5 and D = (1/2) eps_kjl T_l
    gives the rotlet T x r / r^3 (unbounded, times 1 / (8 pi eta))."""
    rng = np.random.default_rng(3)
    x, y = rng.normal(size=3), rng.normal(size=3) + 3
    r = x - y
    rn = np.linalg.norm(r)
    A = rng.normal(size=(3, 3))
    S = 0.5 * (A + A.T) - np.trace(A) / 3 * np.eye(3)
    np.testing.assert_allclose(dipole_flow(oseen_jets(x, y), S), 3 * r * (r @ S @ r) / rn ** 5, rtol=1e-12)
    T = rng.normal(size=3)
    D = wall.force_dipole(np.zeros(5), T, 1.0, 1.0)
    np.testing.assert_allclose(dipole_flow(oseen_jets(x, y), D), np.cross(T, r) / rn ** 3, rtol=1e-12)


def test_stresslet_of_the_active_strain_mode():
    """Far from an active sphere with V^(2s) only, the unbounded superposition velocity is
    the point stresslet flow of S = (20/3) pi eta a^2 V^(2s) (to O(a^2/r^2)), the force
    dipole the sphere exerts on the fluid."""
    a, eta = 1.0, 0.7
    p = np.array([[0.0, 0.6, 0.8], [1.0, 0.0, 0.0]])
    VH = galerkin.active_modes(p, 0.05, 0.0, 2)
    VH[1] = 0.0
    z = np.zeros((2, 3))
    for d in (40.0, 80.0):
        R = np.array([[0.0, 0.0, 0.0], [d, 0.3 * d, -0.2 * d]])
        V, _ = galerkin.superpose(R, z, z, VH, z, z, a, eta, 2)
        S = wall.force_dipole(VH[0], np.zeros(3), a, eta)
        r = R[1] - R[0]
        want = 3 * r * (r @ S @ r) / np.linalg.norm(r) ** 5 / (8 * np.pi * eta)
        assert np.linalg.norm(V[1] - want) < 5 * (a / d) ** 2 * np.linalg.norm(want)


def test_images_fade_far_from_the_wall_and_jets_match_differences():
    rng = np.random.default_rng(4)
    x = np.array([0.4, -0.3, 0.0])
    y = np.array([1.0, 0.5, 0.0])
    mags = []
    for h in (10.0, 100.0, 1000.0):
        W = wall.image_jets(x + [0, 0, h], y + [0, 0, h])
        mags.append(max(abs(w.v) for row in W for w in row))
    assert mags[0] > 8 * mags[1] > 64 * mags[2]
    x, y = random_source(rng), random_source(rng)
    W = wall.image_jets(x, y)
    eps = 1e-5
    for k in range(6):
        dp, dm = np.zeros(6), np.zeros(6)
        dp[k], dm[k] = eps, -eps
        Wp = wall.image_jets(x + dp[:3], y + dp[3:])
        Wm = wall.image_jets(x + dm[:3], y + dm[3:])
        for i in range(3):
            for j in range(3):
                fd = (Wp[i][j].v - Wm[i][j].v) / (2 * eps)
                assert abs(W[i][j].g[k] - fd) < 1e-8 * max(1.0, abs(fd))
                fdg = (Wp[i][j].g - Wm[i][j].g) / (2 * eps)
                assert np.abs(W[i][j].H[k] - fdg).max() < 1e-6 * max(1.0, np.abs(fdg).max())


def test_wall_superposition_reduces_to_the_unbounded_one_far_away():
    rng = np.random.default_rng(5)
    N = 6
    R = rng.normal(size=(N, 3)) * 4
    p = rng.normal(size=(N, 3))
    p /= np.linalg.norm(p, axis=1, keepdims=True)
    VH = galerkin.active_modes(p, 0.05, 0.0, 2)
    Va, Oa = 0.1 * p, np.zeros((N, 3))
    Fe, Te = -0.01 * R, rng.normal(size=(N, 3)) * 0.01
    V0, O0 = galerkin.superpose(R, Va, Oa, VH, Fe, Te, 1.0, 0.7, 2)
    far = R + [0, 0, 1e5]
    V1, O1 = wall.wall_superpose(far, Va, Oa, VH, Fe, Te, 1.0, 0.7)
    np.testing.assert_allclose(V1, V0, atol=1e-6 * np.abs(V0).max())
    np.testing.assert_allclose(O1, O0, atol=1e-6 * np.abs(O0).max())
