"""Flow field of the Galerkin representation at points in the fluid (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module.

Sec. III, Eq. flow_expression / galerkin_representation_flow_yl: the exterior flow is
the single layer of a surface density on every sphere, and (reading R1 of the oracle,
Sec. III Eq. generalized_Qlsigma with Appendix C) the density of sphere m is expanded
in the tensorial harmonics with the flow coefficients Q_m as coefficients,

    q_m(n) = sum_l (2l+1)/(4 pi a^2) Q_m^(l+1) . Y^(l)(n)      (Q^L = F^L),
    v(x)   = -(1/(8 pi eta)) sum_m int_{S_m} G(x - y) . q_m(y) dS_y.

The surface integral is evaluated by a product Gauss-Legendre x trapezoid rule; the
integrand is smooth for x outside every sphere, so the rule converges exponentially
with the distance of x from the surfaces.  Nothing here uses the derivative form of the
pair elements.
"""
import numpy as np

from .galerkin import lower_trial, mode_fields, sphere_rule
from .quadrature import stokeslet
from .tensors import ModeBasis


def internal_coefficients(Fe, Te, QH, a, trunc):
    """x[N][d]: F^L from the external force and torque, then the solved Q^H, in the
    internal coordinates x = c y of every component."""
    MB = ModeBasis(trunc)
    xF = lower_trial(np.asarray(Fe, float), np.asarray(Te, float), a, MB)
    return np.concatenate([xF, np.asarray(QH, float) * MB.scale[MB.nL:]], axis=1)


def flow(X, R, x_int, a, eta, trunc, nt=24, nphi=48):
    """v(X) [M][3] from spheres at R [N][3] with internal coefficients x_int [N][d]."""
    X = np.atleast_2d(np.asarray(X, float))
    R = np.atleast_2d(np.asarray(R, float))
    MB = ModeBasis(trunc)
    pts, wts = sphere_rule(nt, nphi)
    fields = np.stack([mode_fields(E, pts) for E in MB.vectors])          # (d, K, 3)
    pref = (2 * (MB.rank - 1) + 1) / (4 * np.pi * a * a)
    U = np.zeros((len(X), 3))
    for m in range(len(R)):
        q = np.einsum("p,pki->ki", np.asarray(x_int[m], float) * pref, fields)   # density at the nodes
        y = R[m] + a * pts
        G = stokeslet(X[:, None, :] - y[None, :, :])                            # (M, K, 3, 3)
        U -= np.einsum("mkij,k,kj->mi", G, wts * a * a, q) / (8 * np.pi * eta)
    return U
