"""Brute-force surface integrals that pin the oracle (test infrastructure only).

These routines integrate the paper's defining integrals directly, with no use of
the derivative (Taylor) route of ``galerkin.pair_blocks``:

* ``pair_block_bruteforce``: the double surface integral of Sec. III,
  Eq. matrix_elemets_yl (single layer), for two disjoint spheres, by a product
  Gauss-Legendre x trapezoid rule on each sphere (the integrand is smooth, so the
  rule converges exponentially).
* ``self_block_from_flow``: the Galerkin projection onto sphere n's own modes of
  the exterior flow formula of Sec. III, Eq. flow_expression (Appendix B),
  evaluated on the sphere surface where the single layer is continuous.  This is
  an independent route to the self elements of Eq. single_layer_yl_matrix_element.
"""
import numpy as np

from . import taylor
from .galerkin import mode_fields, sphere_rule
from .tensors import ModeBasis


def stokeslet(x):
    """G_ij(x) = delta_ij/|x| + x_i x_j/|x|^3 for x (..., 3)."""
    r = np.linalg.norm(x, axis=-1)
    G = np.eye(3) / r[..., None, None] + x[..., :, None] * x[..., None, :] / (r ** 3)[..., None, None]
    return G


def pair_block_bruteforce(rho, a, trunc, nt=14, nphi=28):
    """<e_p, G_nm e_q> by direct double quadrature for one displacement rho = R_n - R_m."""
    MB = ModeBasis(trunc)
    pts, wts = sphere_rule(nt, nphi)
    fields = np.stack([mode_fields(E, pts) for E in MB.vectors])      # (d, M, 3)
    l = MB.rank - 1
    x = np.asarray(rho, float)[None, None, :] + a * pts[:, None, :] - a * pts[None, :, :]
    G = stokeslet(x)                                                     # (M1, M2, 3, 3)
    Gf = np.einsum("abij,b,qbj->qai", G, wts, fields)                    # (d, M1, 3)
    A = np.einsum("a,pai,qai->pq", wts, fields, Gf)
    pref = np.outer(2 * l + 1, 2 * l + 1) / (16 * np.pi ** 2)
    return A * pref


def self_block_from_flow(a, trunc, nt=14, nphi=28):
    """<e_p, G_nn e_q> from the exterior flow formula evaluated on the surface.

    The single-layer flow of mode q (rank l'+1) of a sphere centred at 0 is
    u_i(x) = a^l' (-1)^l' [F^l' d^(l') G]_{i j beta}(x) e_q[j, beta]  (times -1/(8 pi eta),
    which cancels against the definition of G_nn), with F^l' = 1 + a^2/(4l'+6) lap.
    Projected with (2l+1)/(4 pi a^2) int Y^(l) u dS.
    """
    MB = ModeBasis(trunc)
    pts, wts = sphere_rule(nt, nphi)
    fields = np.stack([mode_fields(E, pts) for E in MB.vectors])      # (d, M, 3)
    Lmax = int(max(MB.rank))
    K = Lmax + 1
    mons = taylor.mono_index(K)
    Dr = taylor.derivatives(a * pts, 1.0, K)
    D1 = taylor.derivatives(a * pts, -1.0, K)

    def dterm(D, mi):
        return D[:, mons[tuple(mi)]]

    d = MB.d
    S = np.zeros((d, d))
    for q in range(d):
        E = MB.vectors[q]
        lq = E.ndim - 1
        c = a * a / (4 * lq + 6)
        u = np.zeros((len(pts), 3))
        # (F G)_ij = 2 delta_ij / r - d_i d_j r - 2 c d_i d_j (1/r)
        for t in np.ndindex(E.shape):
            v = E[t]
            if v == 0.0:
                continue
            j, beta = t[0], t[1:]
            mb = [0, 0, 0]
            for b in beta:
                mb[b] += 1
            for i in range(3):
                mi = list(mb)
                mi[i] += 1
                mi[j] += 1
                val = -dterm(Dr, mi) - 2 * c * dterm(D1, mi)
                if i == j:
                    val = val + 2 * dterm(D1, mb)
                u[:, i] += v * val
        u *= a ** lq * (-1) ** lq
        for p in range(d):
            lp = MB.rank[p] - 1
            S[p, q] = (2 * lp + 1) / (4 * np.pi) * np.sum(wts * np.sum(fields[p] * u, axis=1))
    return S
