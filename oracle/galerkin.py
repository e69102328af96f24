"""Dense Galerkin system of the FP64 CPU oracle (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module.  It restates, in plain dense form, what the paper's method
computes for N spheres of radius a in an unbounded fluid of viscosity eta.

Pair elements (Sec. III, Eq. single_layer_yl_matrix_element, m != n):
    G_nm^(l+1, l'+1) = a^(l+l') F_n^l F_m^l' grad_n^(l) grad_m^(l') G(R_n - R_m),
    F^l = 1 + a^2/(4l+6) lap  (Sec. III, finite-size operator),
with G_ij = (delta_ij lap - d_i d_j) r.  Because grad_m = -grad_rho and
lap lap r = 0 away from the origin,
    (F_n F_m G)_ij = 2 delta_ij / r - d_i d_j r - 2 c d_i d_j (1/r),
    c = a^2 (1/(4l+6) + 1/(4l'+6)).
All derivatives come from ``taylor.derivatives`` (binomial series of |rho+h|^nu).

Self elements (Sec. III, same equation, m = n):
    G_nn^(l+1, l+1) = (2l+1)/(2 pi a) int Y^(l) (I - nn) Y^(l) dOmega,
evaluated by an exact product quadrature; the result is one scalar g per
irreducible mode.

The linear system (reading R1): the rigid-body double layer K^LL = -4 pi I and
K^HL = 0 (Sec. II, text before Eq. many_body_active_passive_VL_FH_relation); for
the higher modes the double layer is carried by the flow coefficients
Q^(l sigma) = F^(l sigma) - c_(l sigma) V^(l sigma) (Sec. III,
Eq. generalized_Qlsigma, Appendix C), which turns the boundary equation into
    8 pi eta V_n = - sum_m G_nm Q_m        (Q^L = F^L)
on every retained mode.  Hence
    G^HH Q^H = -8 pi eta V^H - G^HL F^L,
    8 pi eta V^L = -G^LL F^L - G^LH Q^H,
with F^(1) = -F^e, F^(21) = -T^e/a, V^(1) = V - V^a, V^(21) = 2a (Omega - Omega^a)
(Sec. IV, Eq. stress/velocity multipole embeddings).  The oracle solves the
dense H block by LU with partial pivoting (numpy.linalg.solve).

Superposition (Sec. IV, text before Eq. mobility_matrices, second form): the H
coefficients are replaced by their one-body values, Q^H_m = -8 pi eta V^H_m / g,
and only the direct pair sum remains.

Coordinates: every mode component is stored as x = c * y where y is the packed
coordinate (``tensors.stf_basis``) of the paper's irreducible tensor and c the
norm of its embedding (``tensors.ModeBasis``); in x the operator is symmetric.
"""
import math
from functools import lru_cache

import numpy as np

from . import taylor
from .tensors import ModeBasis, dfact, tsh


# ----------------------------------------------------------------------------
# polynomial forms of the mode tensors
# ----------------------------------------------------------------------------

def _poly_coeffs(E, K):
    """Coefficients over monomials(K) of sum_t E[t] x^t for a full tensor E."""
    idx = taylor.mono_index(K)
    out = np.zeros(len(idx))
    if E.ndim == 0:
        out[0] = float(E)
        return out
    for t in np.ndindex(E.shape):
        v = E[t]
        if v != 0.0:
            n = [0, 0, 0]
            for i in t:
                n[i] += 1
            out[idx[tuple(n)]] += v
    return out


def _poly_mul(A, B, K):
    return taylor.mul(A[None, :], B[None, :], K)[0]


@lru_cache(maxsize=None)
def _pair_weights(trunc, a):
    """Matrices Wr, W1 with block[p, q] = Wr @ d^n r + W1 @ d^n (1/r)."""
    MB = ModeBasis(trunc)
    Lmax = max(MB.rank)
    K = 2 * Lmax
    nm = len(taylor.monomials(K))
    polys, vpolys = [], []
    for E in MB.vectors:
        polys.append(_poly_coeffs(E, K))
        vpolys.append([_poly_coeffs(E[i], K) for i in range(3)])
    d = MB.d
    Wr = np.zeros((d, d, nm))
    W1 = np.zeros((d, d, nm))
    for p in range(d):
        lp = MB.rank[p] - 1
        for q in range(d):
            lq = MB.rank[q] - 1
            pref = a ** (lp + lq) * (-1) ** lq
            c = a * a * (1.0 / (4 * lp + 6) + 1.0 / (4 * lq + 6))
            W = _poly_mul(polys[p], polys[q], K)
            Wd = sum(_poly_mul(vpolys[p][i], vpolys[q][i], K) for i in range(3))
            Wr[p, q] = -pref * W
            W1[p, q] = pref * (2.0 * Wd - 2.0 * c * W)
    return Wr.reshape(d * d, nm), W1.reshape(d * d, nm), K, d


def pair_blocks(rho, a, trunc):
    """G_nm for displacement(s) rho = R_n - R_m: array (P, d, d) in x coordinates."""
    rho = np.atleast_2d(np.asarray(rho, float))
    Wr, W1, K, d = _pair_weights(trunc, float(a))
    out = np.empty((rho.shape[0], d, d))
    chunk = 2048
    for s in range(0, rho.shape[0], chunk):
        r = rho[s:s + chunk]
        Dr = taylor.derivatives(r, 1.0, K)
        D1 = taylor.derivatives(r, -1.0, K)
        out[s:s + chunk] = (Dr @ Wr.T + D1 @ W1.T).reshape(-1, d, d)
    return out


# ----------------------------------------------------------------------------
# self elements by quadrature
# ----------------------------------------------------------------------------

def sphere_rule(nt, nphi):
    """Gauss-Legendre (cos theta) x uniform (phi) rule: points (M,3), weights (M,)."""
    x, w = np.polynomial.legendre.leggauss(nt)
    phi = 2 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1 - x * x)
    pts = np.stack([np.outer(st, np.cos(phi)), np.outer(st, np.sin(phi)),
                    np.outer(x, np.ones(nphi))], axis=-1).reshape(-1, 3)
    wts = np.outer(w, np.full(nphi, 2 * np.pi / nphi)).reshape(-1)
    return pts, wts


def mode_fields(E, pts):
    """(E . Y^(l))(n)_i = sum_alpha E[i, alpha] Y^(l)_alpha(n) at the points: (M, 3)."""
    L = E.ndim
    l = L - 1
    out = np.zeros((len(pts), 3))
    for k, n in enumerate(pts):
        Y = tsh(l, n)
        out[k] = np.tensordot(E, Y, axes=l) if l > 0 else E * Y
    return out


@lru_cache(maxsize=None)
def self_matrix(trunc, a):
    """<e_p, G_nn e_q> for all component pairs (d, d); block-diagonal by rank L."""
    MB = ModeBasis(trunc)
    pts, wts = sphere_rule(12, 26)
    fields = [mode_fields(E, pts) for E in MB.vectors]
    d = MB.d
    S = np.zeros((d, d))
    for p in range(d):
        for q in range(d):
            if MB.rank[p] != MB.rank[q]:
                continue
            l = MB.rank[p] - 1
            fp, fq = fields[p], fields[q]
            integrand = np.sum(fp * fq, axis=1) - np.sum(fp * pts, axis=1) * np.sum(fq * pts, axis=1)
            S[p, q] = (2 * l + 1) / (2 * np.pi * a) * np.sum(wts * integrand)
    return S


def self_scalars(trunc, a):
    """One scalar g per component (diagonal of ``self_matrix``)."""
    return np.diag(self_matrix(trunc, a)).copy()


# ----------------------------------------------------------------------------
# user coordinates <-> internal x coordinates
# ----------------------------------------------------------------------------

def vec_to_packed(v):
    """Cartesian vectors (..., 3) -> packed rank-1 coordinates (mu = -1, 0, 1 -> y, z, x)."""
    v = np.asarray(v, float)
    return v[..., [1, 2, 0]]


def packed_to_vec(y):
    y = np.asarray(y, float)
    return y[..., [2, 0, 1]]


def lower_trial(Fe, Te, a, MB):
    """x coordinates of F^L from external force and torque: (N, 6)."""
    x1 = vec_to_packed(-np.asarray(Fe, float))
    x2 = vec_to_packed(-np.asarray(Te, float) / a) * MB.scale[3]
    return np.concatenate([x1, x2], axis=1)


def lower_velocity(xL, Va, Oa, a, MB):
    """V, Omega from x coordinates of V^L (N, 6)."""
    V = np.asarray(Va, float) + packed_to_vec(xL[:, 0:3])
    Om = np.asarray(Oa, float) + packed_to_vec(xL[:, 3:6] / MB.scale[3] / (2 * a))
    return V, Om


# ----------------------------------------------------------------------------
# dense system
# ----------------------------------------------------------------------------

def ordered_pairs(N):
    n, m = np.nonzero(~np.eye(N, dtype=bool))
    return n, m


def assemble(R, a, trunc):
    """Full dense G (N*d, N*d) in x coordinates, particle-major."""
    R = np.asarray(R, float)
    N = R.shape[0]
    MB = ModeBasis(trunc)
    d = MB.d
    A = np.zeros((N, d, N, d))
    n, m = ordered_pairs(N)
    if len(n):
        blocks = pair_blocks(R[n] - R[m], a, trunc)
        A[n, :, m, :] = blocks
    g = self_scalars(trunc, a)
    for i in range(N):
        A[i, :, i, :] = np.diag(g)
    return A.reshape(N * d, N * d)


def solve(R, Va, Oa, VH, Fe, Te, a, eta, trunc, return_all=False):
    """Galerkin solve by dense LU.  Returns V, Omega (N,3) and Q^H packed (N,h)."""
    R = np.asarray(R, float)
    N = R.shape[0]
    MB = ModeBasis(trunc)
    d, nL, h = MB.d, MB.nL, MB.h
    A = assemble(R, a, trunc).reshape(N, d, N, d)
    xF = lower_trial(Fe, Te, a, MB)                              # (N, 6)
    xVH = np.asarray(VH, float).reshape(N, h) * MB.scale[nL:]    # (N, h)
    AHH = A[:, nL:, :, nL:].reshape(N * h, N * h)
    AHL = A[:, nL:, :, :nL].reshape(N * h, N * nL)
    ALL = A[:, :nL, :, :nL].reshape(N * nL, N * nL)
    ALH = A[:, :nL, :, nL:].reshape(N * nL, N * h)
    b = -8 * np.pi * eta * xVH.reshape(-1) - AHL @ xF.reshape(-1)
    xQ = np.linalg.solve(AHH, b) if h else np.zeros(0)
    xVL = -(ALL @ xF.reshape(-1) + ALH @ xQ) / (8 * np.pi * eta)
    V, Om = lower_velocity(xVL.reshape(N, nL), Va, Oa, a, MB)
    QH = xQ.reshape(N, h) / MB.scale[nL:]
    if return_all:
        return V, Om, QH, dict(A=A, b=b, xQ=xQ, xF=xF, AHH=AHH)
    return V, Om, QH


def one_body_QH(VH, a, eta, trunc):
    """Isolated-sphere flow coefficients Q^H = -8 pi eta V^H / g (packed, paper normalisation)."""
    MB = ModeBasis(trunc)
    g = self_scalars(trunc, a)[MB.nL:]
    return -8 * np.pi * eta * np.asarray(VH, float) / g


def superpose(R, Va, Oa, VH, Fe, Te, a, eta, trunc=2, targets=None):
    """Superposition approximation: one-body Q^H, direct pair sum for V, Omega.

    ``targets`` (optional index array) restricts the outputs to those spheres."""
    R = np.asarray(R, float)
    N = R.shape[0]
    MB = ModeBasis(trunc)
    d, nL, h = MB.d, MB.nL, MB.h
    tgt = np.arange(N) if targets is None else np.asarray(targets)
    x = np.zeros((N, d))
    x[:, :nL] = lower_trial(Fe, Te, a, MB)
    x[:, nL:] = one_body_QH(VH, a, eta, trunc) * MB.scale[nL:]
    y = apply_offdiag(R, x, a, trunc, rows=slice(0, nL), targets=tgt)
    g = self_scalars(trunc, a)
    xVL = -(y + g[:nL] * x[tgt, :nL]) / (8 * np.pi * eta)
    return lower_velocity(xVL, np.asarray(Va, float)[tgt], np.asarray(Oa, float)[tgt], a, MB)


def apply_offdiag(R, x, a, trunc, rows=slice(None), targets=None):
    """y_n = sum_{m != n} G_nm x_m (x coordinates), optionally for a subset of targets/rows."""
    R = np.asarray(R, float)
    N = R.shape[0]
    x = np.asarray(x, float)
    tgt = np.arange(N) if targets is None else np.asarray(targets)
    MB = ModeBasis(trunc)
    d = MB.d
    out = np.zeros((len(tgt), d))
    for k, n in enumerate(tgt):
        m = np.array([j for j in range(N) if j != n])
        if len(m) == 0:
            continue
        blocks = pair_blocks(R[n] - R[m], a, trunc)         # (N-1, d, d)
        out[k] = np.einsum("mpq,mq->p", blocks, x[m])
    return out[:, rows]


# ----------------------------------------------------------------------------
# user-facing helpers for the trap workloads
# ----------------------------------------------------------------------------

def active_modes(p, s0, d0, trunc):
    """Packed V^H for the uniaxial trap parametrisation (Sec. V):
    V^(20) = s0 (pp - I/3), V^(32) = d0 p, every other H mode zero."""
    from .tensors import pack_stf
    p = np.asarray(p, float)
    MB = ModeBasis(trunc)
    out = np.zeros((p.shape[0], MB.h))
    for n in range(p.shape[0]):
        S = s0 * (np.outer(p[n], p[n]) - np.eye(3) / 3)
        out[n, 0:5] = pack_stf(S)
        out[n, 5:8] = vec_to_packed(d0 * p[n])
    return out
