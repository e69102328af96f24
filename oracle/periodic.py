"""Spheres in a periodic cube: the superposition approximation with the periodic
Green's function, summed by Ewald's method (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module.

Sec. VI: in a periodic domain the flow summation is only conditionally convergent and a
limiting procedure fixes it; here that is Hasimoto's: the mean flow over the cell is
zero (the k = 0 term is left out, a uniform pressure gradient balancing the net force).
With G = (d_ij lap - d_i d_j) r the Oseen tensor (u = G F / (8 pi eta)), Ewald's split
r = r erfc(xi r) + r erf(xi r) gives

    G^real_ij(r) = d_ij (f'' + f'/r) - (f'' - f'/r) r_i r_j / r^2,   f = r erfc(xi r),
    G^rec(k)    = 8 pi (d - k k / k^2) / k^2 (1 + k^2/(4 xi^2) + k^4/(8 xi^4)) exp(-k^2/(4 xi^2)),
    G^per(x)    = sum_n G^real(x + n L) + (1/L^3) sum_{k != 0} G^rec(k) cos(k.x),

k = 2 pi m / L (the Fourier transform of r erf(xi r) is -8 pi / k^4 times the bracket and
the Gaussian).  A sphere's own periodic images (x -> 0, the singular direct term left
out) give G^per_self = sum_{n != 0} G^real(n L) + (1/L^3) sum_{k != 0} G^rec(k)
- (8 xi / sqrt(pi)) I, the last term being the limit of G - G^real at r = 0.

The superposition of Sec. IV in the periodic cube (reading of this build), at the
point-force level: V_n = V^a_n + F_n / (6 pi eta a) + [sum_{m != n} G^per(R_n - R_m) F_m
+ G^per_self F_n] / (8 pi eta).  Force dipoles, the finite-size terms and the rotation
rates are not included.  The sums here are direct (every lattice vector and wave vector
up to the cut-offs); nothing about the result depends on xi, which the tests pin.
"""
import math

import numpy as np
from scipy.special import erfc


def real_tensor(r, xi):
    """G^real(r) for separations r (..., 3), r != 0: (..., 3, 3)."""
    r = np.asarray(r, float)
    rn = np.linalg.norm(r, axis=-1)
    e = np.exp(-(xi * rn) ** 2)
    f1 = erfc(xi * rn) - 2 * xi * rn / math.sqrt(math.pi) * e
    f2 = 4 * xi / math.sqrt(math.pi) * ((xi * rn) ** 2 - 1) * e
    rh = r / rn[..., None]
    a = f2 + f1 / rn
    b = f2 - f1 / rn
    return a[..., None, None] * np.eye(3) - b[..., None, None] * rh[..., :, None] * rh[..., None, :]


def lattice(L, nmax):
    g = np.arange(-nmax, nmax + 1)
    n = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    return n * L


def recip_tensors(L, xi, mmax):
    """Wave vectors k != 0 with |m_i| <= mmax and G^rec(k) / L^3."""
    g = np.arange(-mmax, mmax + 1)
    m = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    m = m[np.any(m != 0, axis=1)]
    k = 2 * math.pi * m / L
    k2 = (k * k).sum(1)
    q = k2 / (4 * xi * xi)
    pref = 8 * math.pi / k2 * (1 + q + 2 * q * q) * np.exp(-q) / L ** 3
    kk = k[:, :, None] * k[:, None, :] / k2[:, None, None]
    return k, pref[:, None, None] * (np.eye(3) - kk)


def periodic_tensor(x, L, xi, nmax=3, mmax=8):
    """G^per(x) for x not on the lattice (x: (3,)).  G^per is L-periodic and the lattice
    sum below is truncated, so x is first reduced to its nearest image."""
    x = np.asarray(x, float)
    x = x - L * np.rint(x / L)
    n = lattice(L, nmax)
    G = real_tensor(x + n, xi).sum(0)
    k, Gk = recip_tensors(L, xi, mmax)
    return G + (Gk * np.cos(k @ x)[:, None, None]).sum(0)


def periodic_tensors(X, L, xi, nmax=3, mmax=8, chunk=256):
    """G^per(x) for many separations X (M, 3) (none on the lattice): (M, 3, 3)."""
    X = np.atleast_2d(np.asarray(X, float))
    X = X - L * np.rint(X / L)                 # nearest images (G^per is L-periodic)
    n = lattice(L, nmax)
    k, Gk = recip_tensors(L, xi, mmax)
    out = np.zeros((len(X), 3, 3))
    for c0 in range(0, len(X), chunk):
        x = X[c0:c0 + chunk]
        out[c0:c0 + chunk] = real_tensor(x[:, None, :] + n[None], xi).sum(1)
        out[c0:c0 + chunk] += np.einsum("km,kij->mij", np.cos(k @ x.T), Gk)
    return out


def self_tensor(L, xi, nmax=3, mmax=8):
    """G^per_self: a point force's own periodic images at its position."""
    n = lattice(L, nmax)
    n = n[np.any(n != 0, axis=1)]
    G = real_tensor(n, xi).sum(0)
    _, Gk = recip_tensors(L, xi, mmax)
    return G + Gk.sum(0) - 8 * xi / math.sqrt(math.pi) * np.eye(3)


def periodic_superpose(R, Va, Fe, a, eta, L, xi=None, targets=None, nmax=3, mmax=8):
    """V (targets, 3) of the point-force superposition in the periodic cube of side L."""
    R = np.asarray(R, float)
    Fe = np.asarray(Fe, float)
    xi = 5.0 / L if xi is None else xi
    tg = np.arange(len(R)) if targets is None else np.asarray(targets)
    S = self_tensor(L, xi, nmax, mmax)
    V = np.asarray(Va, float)[tg] + Fe[tg] / (6 * math.pi * eta * a)
    for q, n in enumerate(tg):
        others = np.arange(len(R)) != n
        G = periodic_tensors(R[n] - R[others], L, xi, nmax, mmax)
        u = S @ Fe[n] + np.einsum("mij,mj->i", G, Fe[others])
        V[q] += u / (8 * math.pi * eta)
    return V
