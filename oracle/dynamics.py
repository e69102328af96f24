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
