"""Spheres above a plane no-slip wall: the superposition approximation with the wall's
Green's function (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module.

Sec. VI: the method extends to other geometries by using the Green's function of
that geometry in the boundary integrals.  For a plane wall z = 0 (fluid z > 0) that is
Blake's solution: the Oseen tensor plus an image system at y* = (y1, y2, -y3),

    G^B_ij(x, y) = G_ij(x - y) + W_ij(x, y),
    W_ij = -G_ij(R) + 2h m_j [ h (d_ij/|R|^3 - 3 R_i R_j/|R|^5) + d_i3 R_j/|R|^3
                               - (d_ij R_3 + R_i d_j3)/|R|^3 + 3 R_i R_3 R_j/|R|^5 ],
    R = x - y*,  h = y3,  m = (1, 1, -1),

so that the flow of a point force F at y is u = G^B F / (8 pi eta) and vanishes on the
wall.  The superposition of Sec. IV near the wall (reading of this build): every sphere
keeps the unbounded direct pair terms of galerkin.superpose, and the image flow of its
force, torque and stresslet -- at the point-singularity level -- is added at every
sphere centre, its own included:

    u_img(x) = [ W_ij(x, y) F_j + D_jk d/dy_k W_ij(x, y) ] / (8 pi eta),  y = R_m,
    D_jk = S_jk + (1/2) eps_kjl T_l,   S = (20/3) pi eta a^2 V^(2s),
    V_n += u_img(R_n),   Omega_n += (1/2) curl u_img (R_n).

F, T and S are what the sphere exerts on the fluid: its external force and torque, and
the force dipole -a Q^(2s) of its one-body traction (Q^(2s) = -(20/3) pi eta a V^(2s),
Table III C20; a squirmer's -4 pi eta a^2 B2 (pp - I/3)).  (The dipole tensor D gives the
stresslet flow 3 r (r.S.r) / (8 pi eta r^5) and the rotlet T x r / (8 pi eta r^3) in the
unbounded part, pinned in the tests.)  The image flows of
the potential dipole V^(3t) and the finite-size (a^2) terms of the images are left out.

Derivatives with respect to x and y are taken exactly (to rounding) by forward-mode
differentiation: `Jet` carries a value with its gradient and Hessian in the six
variables (x, y), for a batch of points at once (leading axis).
"""
import numpy as np

from .galerkin import superpose
from .tensors import unpack_stf

M_DIAG = np.array([1.0, 1.0, -1.0])
LEVI = np.zeros((3, 3, 3))
for (i, j, k), s in {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1,
                     (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}.items():
    LEVI[i, j, k] = s


def _outer(a, b):
    return a[..., :, None] * b[..., None, :]


class Jet:
    """Values with their gradients (..., 6) and Hessians (..., 6, 6) in the variables
    (x, y); the leading shape is a batch of independent points (or none)."""

    __slots__ = ("v", "g", "H")

    def __init__(self, v, g=None, H=None):
        self.v = np.asarray(v, float)
        self.g = np.zeros(self.v.shape + (6,)) if g is None else g
        self.H = np.zeros(self.v.shape + (6, 6)) if H is None else H

    @staticmethod
    def var(v, k):
        v = np.asarray(v, float)
        g = np.zeros(v.shape + (6,))
        g[..., k] = 1.0
        return Jet(v, g)

    def _c(self, o):
        return o if isinstance(o, Jet) else Jet(np.broadcast_to(np.asarray(o, float), self.v.shape))

    def __add__(self, o):
        o = self._c(o)
        return Jet(self.v + o.v, self.g + o.g, self.H + o.H)

    __radd__ = __add__

    def __neg__(self):
        return Jet(-self.v, -self.g, -self.H)

    def __sub__(self, o):
        return self + (-self._c(o))

    def __rsub__(self, o):
        return self._c(o) - self

    def __mul__(self, o):
        o = self._c(o)
        sv, ov = self.v[..., None], o.v[..., None]
        return Jet(self.v * o.v, sv * o.g + ov * self.g,
                   sv[..., None] * o.H + ov[..., None] * self.H + _outer(self.g, o.g) + _outer(o.g, self.g))

    __rmul__ = __mul__

    def _chain(self, f0, f1, f2):
        """f(self) for f with f(v) = f0, f'(v) = f1, f''(v) = f2."""
        f1, f2 = np.asarray(f1)[..., None], np.asarray(f2)[..., None]
        return Jet(f0, f1 * self.g, f1[..., None] * self.H + f2[..., None] * _outer(self.g, self.g))

    def inv(self):
        v = self.v
        return self._chain(1.0 / v, -1.0 / v ** 2, 2.0 / v ** 3)

    def __truediv__(self, o):
        return self * self._c(o).inv()

    def sqrt(self):
        s = np.sqrt(self.v)
        return self._chain(s, 0.5 / s, -0.25 / (s * self.v))


def image_tensor(xj, yj):
    """W_ij(x, y) (3 x 3 of Jets) from Jet coordinates x (3) and y (3)."""
    R = [xj[0] - yj[0], xj[1] - yj[1], xj[2] + yj[2]]
    h = yj[2]
    R2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2]
    iR = R2.sqrt().inv()
    iR3 = iR * iR * iR
    iR5 = iR3 * iR * iR
    W = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            d = 1.0 if i == j else 0.0
            g = d * iR + R[i] * R[j] * iR3                    # Oseen tensor at R
            t = h * (d * iR3 - 3.0 * R[i] * R[j] * iR5)
            if i == 2:
                t = t + R[j] * iR3
            t = t - (d * R[2] + (R[i] if j == 2 else 0.0)) * iR3
            t = t + 3.0 * R[i] * R[2] * R[j] * iR5
            W[i][j] = -g + 2.0 * M_DIAG[j] * h * t
    return W


def image_jets(x, y):
    """W_ij at (x, y) with derivatives: Jets in the variables (x_0..2, y_0..2).  x and y
    are points (3,) or batches (M, 3) (broadcast against each other)."""
    x, y = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float))
    xj = [Jet.var(x[..., k], k) for k in range(3)]
    yj = [Jet.var(y[..., k], 3 + k) for k in range(3)]
    return image_tensor(xj, yj)


def blake(x, y):
    """Full wall Green's function G^B_ij(x, y) (Oseen + images), values only."""
    r = np.asarray(x, float) - np.asarray(y, float)
    rn = np.linalg.norm(r)
    G = np.eye(3) / rn + np.outer(r, r) / rn ** 3
    W = image_jets(x, y)
    return G + np.array([[W[i][j].v for j in range(3)] for i in range(3)])


def image_velocity(x, y, F, D):
    """Image flow at x (times 8 pi eta) of forces F (..., 3) and force dipoles D (..., 3, 3)
    at y, and its vorticity (curl): (u (..., 3), curl u (..., 3)) per source."""
    W = image_jets(x, y)
    F, D = np.asarray(F, float), np.asarray(D, float)
    shape = W[0][0].v.shape
    u = np.zeros(shape + (3,))
    du = np.zeros(shape + (3, 3))          # du[..., i, l] = d u_i / d x_l
    for i in range(3):
        for j in range(3):
            w = W[i][j]
            u[..., i] += w.v * F[..., j] + np.einsum("...k,...k->...", D[..., j, :], w.g[..., 3:])
            du[..., i, :] += w.g[..., :3] * F[..., j, None] + np.einsum("...lk,...k->...l", w.H[..., :3, 3:],
                                                                         D[..., j, :])
    curl = np.stack([du[..., 2, 1] - du[..., 1, 2], du[..., 0, 2] - du[..., 2, 0], du[..., 1, 0] - du[..., 0, 1]],
                    axis=-1)
    return u, curl


def force_dipole(VH, Te, a, eta):
    """D_jk = S_jk + (1/2) eps_kjl T_l with S = (20/3) pi eta a^2 V^(2s)."""
    S = (20.0 / 3.0) * np.pi * eta * a * a * unpack_stf(np.asarray(VH, float)[:5], 2)
    return S + 0.5 * np.einsum("kjl,l->jk", LEVI, np.asarray(Te, float))


def wall_superpose(R, Va, Oa, VH, Fe, Te, a, eta, targets=None):
    """Superposition near the wall z = 0: the unbounded l <= 2 superposition plus the
    image flows of every sphere's force, torque and stresslet (its own included)."""
    R = np.asarray(R, float)
    N = len(R)
    tg = np.arange(N) if targets is None else np.asarray(targets)
    V, Om = superpose(R, Va, Oa, VH, Fe, Te, a, eta, 2, targets=targets)
    D = np.array([force_dipole(VH[m], Te[m], a, eta) for m in range(N)])
    Fe = np.asarray(Fe, float)
    for k, n in enumerate(tg):
        du, dc = image_velocity(R[n], R, Fe, D)         # every source m at once
        V[k] += du.sum(axis=0) / (8 * np.pi * eta)
        Om[k] += 0.5 * dc.sum(axis=0) / (8 * np.pi * eta)
    return V, Om
