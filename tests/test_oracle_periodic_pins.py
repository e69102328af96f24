"""Pins of the periodic oracle (oracle/periodic.py) against what the mathematics fixes.

* the Ewald split: nothing depends on the splitting parameter xi, and the real-space
  tensor plus the reciprocal one is the Oseen tensor (checked through xi-independence of
  lattice sums that converge for every xi);
* Hasimoto (1959): a point force's own periodic images in a simple cubic lattice of side
  L slow it by the factor 1 - 2.837297 a / L (G^per_self = -(4/3) 2.837297 / L I);
* a simple cubic array in a box holding 2 x 2 x 2 of its cells moves exactly like the
  array of one sphere per cell (the pair terms agree with the self term);
* G^per is even and periodic, and its regular part is continuous at the origin.
"""
import math

import numpy as np
import pytest

from oracle import periodic as P


def test_xi_independence():
    L = 10.0
    x = np.array([1.3, -2.1, 0.7])
    ref = P.periodic_tensor(x, L, 0.5, nmax=4, mmax=14)
    for xi in (0.3, 0.8):
        np.testing.assert_allclose(P.periodic_tensor(x, L, xi, nmax=4, mmax=14), ref, atol=1e-12)
        np.testing.assert_allclose(P.self_tensor(L, xi, nmax=4, mmax=14), P.self_tensor(L, 0.5, nmax=4, mmax=14),
                                   atol=1e-12)


@pytest.mark.parametrize("L", [5.0, 12.0])
def test_hasimoto_self_mobility(L):
    S = P.self_tensor(L, 6.0 / L, nmax=3, mmax=12)
    np.testing.assert_allclose(S, -(4.0 / 3.0) * 2.837297 / L * np.eye(3), rtol=2e-7, atol=1e-14 / L)


def test_supercell_of_a_simple_cubic_array():
    L, a, eta = 4.0, 1.0, 0.7
    g = np.arange(2) * L
    R = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 0.3
    F = np.tile([0.2, -0.1, 0.5], (8, 1))
    z = np.zeros((8, 3))
    V8 = P.periodic_superpose(R, z, F, a, eta, 2 * L, nmax=3, mmax=14)
    V1 = P.periodic_superpose(R[:1], z[:1], F[:1], a, eta, L, nmax=3, mmax=14)
    np.testing.assert_allclose(V8, np.tile(V1, (8, 1)), rtol=1e-11)
    want = F[0] / (6 * np.pi * eta * a) * (1 - 2.837297 * a / L)
    np.testing.assert_allclose(V1[0], want, rtol=1e-6)      # the constant is known to 7 digits


def test_even_periodic_and_regular_at_the_origin():
    L, xi = 7.0, 0.6
    rng = np.random.default_rng(3)
    for _ in range(5):
        x = rng.uniform(-L / 2, L / 2, size=3)
        G = P.periodic_tensor(x, L, xi)
        np.testing.assert_allclose(P.periodic_tensor(-x, L, xi), G, atol=1e-13)
        np.testing.assert_allclose(P.periodic_tensor(x + [0.0, L, 0.0], L, xi), G, atol=1e-12)
        np.testing.assert_allclose(P.periodic_tensor(x + [3 * L, -4 * L, 5 * L], L, xi), G, atol=1e-12)
    S = P.self_tensor(L, xi)
    for eps in (1e-3, 1e-4):
        x = eps * np.array([0.3, -0.5, 0.8])
        r = np.linalg.norm(x)
        reg = P.periodic_tensor(x, L, xi) - (np.eye(3) / r + np.outer(x, x) / r ** 3)
        assert np.abs(reg - S).max() < 50 * eps / L ** 2
