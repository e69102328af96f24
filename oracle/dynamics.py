"""Forward-Euler rigid-body and trap update of the oracle (test infrastructure only).

Kinematics (Sec. II): dR/dt = V, dp/dt = Omega x p.  Trap (Sec. V, Eq. trap_eom):
F^e = -k R, T^e = 0, V^a = v_s p, V^(2s) = s0 (pp - I/3), V^(3t) = d0 p.
Reading: every step re-evaluates V, Omega at the current state and renormalises p.
"""
import numpy as np

from . import galerkin


def trap_inputs(R, p, prm, trunc):
    R = np.asarray(R, float)
    p = np.asarray(p, float)
    N = R.shape[0]
    return dict(Va=prm["vs"] * p, Oa=np.zeros((N, 3)),
                VH=galerkin.active_modes(p, prm["s0"], prm["d0"], trunc),
                Fe=-prm["k"] * R, Te=np.zeros((N, 3)))


def velocities(R, p, prm, trunc, superposition):
    inp = trap_inputs(R, p, prm, trunc)
    if superposition:
        return galerkin.superpose(R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"],
                                  prm["a"], prm["eta"], trunc)
    V, Om, _ = galerkin.solve(R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"],
                              prm["a"], prm["eta"], trunc)
    return V, Om


def euler(R, p, V, Om, dt):
    Rn = np.asarray(R, float) + dt * np.asarray(V, float)
    pn = np.asarray(p, float) + dt * np.cross(Om, p)
    pn /= np.linalg.norm(pn, axis=1, keepdims=True)
    return Rn, pn


def trajectory(R, p, prm, trunc, dt, steps, superposition=False):
    for _ in range(steps):
        V, Om = velocities(R, p, prm, trunc, superposition)
        R, p = euler(R, p, V, Om, dt)
    return R, p


def squirmer_slip(p, B1, B2, n):
    """Active slip of a squirmer (Sec. V, Lighthill-Blake, first two modes) at unit surface
    normals n [K][3]: v^a = (n n - I) . [B1 p + B2 (p p - I/3) . n]."""
    p = np.asarray(p, float)
    n = np.atleast_2d(np.asarray(n, float))
    S = np.outer(p, p) - np.eye(3) / 3
    w = B1 * p[None, :] + (n @ S.T) * B2
    return n * np.sum(n * w, axis=1, keepdims=True) - w


def squirmer_modes(p, B1, B2, trunc, nt=16, nphi=32):
    """(V^a, Omega^a, packed V^H) of one squirmer: the slip's tensorial-harmonic
    coefficients V^(l+1) = (2l+1) <v^a (x) Y^(l)> (Sec. III, velocity expansion and the
    orthogonality of the Y^(l)), split into the irreducible modes of the truncation by the
    mode basis (V^(lsigma) packed coordinates y = <e, V^(l+1)> / c), with V^a = -<v^a>
    and Omega^a from the antisymmetric rank-2 part (zero for this axisymmetric slip)."""
    from .galerkin import sphere_rule
    from .tensors import ModeBasis, tsh
    MB = ModeBasis(trunc)
    pts, wts = sphere_rule(nt, nphi)
    v = squirmer_slip(p, B1, B2, pts)                      # (K, 3)
    wn = wts / wts.sum()
    coeff = {}
    for L in sorted({m[1] for m in MB.modes}):
        l = L - 1
        Y = np.stack([tsh(l, n) for n in pts]) if l > 0 else np.ones(len(pts))
        coeff[L] = (2 * l + 1) * np.tensordot(wn[:, None] * v, Y, axes=([0], [0]))
    y = np.array([np.sum(e * coeff[MB.rank[i]]) / MB.scale[i] for i, e in enumerate(MB.vectors)])
    Va = -coeff[1]
    # 2a packed (y, z, x) coordinates hold the antisymmetric rank-2 part
    Oa_packed = y[3:6]
    return Va, Oa_packed, y[MB.nL:]
