"""Superposition above a plane no-slip wall (gbi_wall_superpose) against the oracle.

The oracle (oracle/wall.py, pinned by no slip on the wall, reciprocity, the classical
wall mobilities of a point force and the wall velocity and turning of a pusher) adds the
image flows of every sphere's force, torque and stresslet to the unbounded
superposition, differentiating Blake's image system by forward-mode jets; the GPU does
the same with its own nested dual numbers.  FP64 to 1e-12 of the largest output,
FP32 to 1e-5 (the pair-velocity bar); the N = 10^4 trap cloud above the wall at sampled
spheres.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle import dynamics, galerkin, wall

pytestmark = pytest.mark.gpu


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


def cloud_above_wall(N, seed, zmin=1.4):
    s = workloads.small_cloud(N, seed, phi=0.05)
    R = s["R"].copy()
    R[:, 2] += zmin * s["a"] - R[:, 2].min()
    prm = dict(a=s["a"], eta=s["eta"], k=s["k"], vs=s["vs"], s0=s["s0"], d0=0.0)
    inp = dynamics.trap_inputs(R, s["p"], prm, 2)
    inp["Te"] = np.random.default_rng(seed).normal(size=(N, 3)) * 0.01
    return R, s, inp


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_wall_superposition_matches_oracle(ctx, gbi, precision, tol):
    R, s, inp = cloud_above_wall(40, 71)
    V_o, O_o = wall.wall_superpose(R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"], s["a"], s["eta"])
    prm = gbi.params(a=s["a"], eta=s["eta"], trunc=2, precision=precision)
    t = {k: dev(v) for k, v in inp.items()}
    V, O = ctx.wall_superpose(prm, dev(R), t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"])
    torch.cuda.synchronize()
    assert np.abs(V.cpu().numpy() - V_o).max() <= tol * np.abs(V_o).max()
    assert np.abs(O.cpu().numpy() - O_o).max() <= tol * np.abs(O_o).max()
    # the wall's own contribution is far above the tolerance (the comparison means something)
    V_u, O_u = galerkin.superpose(R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"], s["a"], s["eta"], 2)
    assert np.abs(V_o - V_u).max() > 100 * tol * np.abs(V_o).max()


def test_pusher_near_the_wall_on_the_gpu(ctx, gbi):
    """One pusher (V^(2s) with s0 > 0 exerts S = (20/3) pi eta a^2 s0 (pp - I/3) on the fluid)
    at height h, p at angle theta to the wall: the wall-normal velocity and the turning
    rate of the oracle's Berke pins, through the GPU path."""
    a, eta, s0, h = 1.0, 1.0 / (6 * math.pi), 0.05, 4.0
    p_str = (20.0 / 3.0) * math.pi * eta * a * a * s0
    for theta in (0.0, 0.4, 1.1):
        p = np.array([[math.cos(theta), 0.0, math.sin(theta)]])
        R = np.array([[0.3, -0.2, h]])
        VH = galerkin.active_modes(p, s0, 0.0, 2)
        z = np.zeros((1, 3))
        prm = gbi.params(a=a, eta=eta, trunc=2, precision=0)
        V, O = ctx.wall_superpose(prm, dev(R), dev(z), dev(z), dev(VH), dev(z), dev(z))
        torch.cuda.synchronize()
        V, O = V.cpu().numpy()[0], O.cpu().numpy()[0]
        uz = -3 * p_str * (1 - 3 * math.sin(theta) ** 2) / (64 * math.pi * eta * h ** 2)
        assert V[2] == pytest.approx(uz, rel=1e-12, abs=1e-16)
        thdot = np.cross(O, p[0])
        want = -3 * p_str * math.sin(theta) * math.cos(theta) / (64 * math.pi * eta * h ** 3)
        got = thdot[2] / math.cos(theta)
        assert got == pytest.approx(want, rel=1e-12, abs=1e-16)


def test_wall_fades_far_away(ctx, gbi):
    R, s, inp = cloud_above_wall(30, 72)
    R = R + [0.0, 0.0, 1e6]
    prm = gbi.params(a=s["a"], eta=s["eta"], trunc=2, precision=0)
    t = {k: dev(v) for k, v in inp.items()}
    Vw, Ow = ctx.wall_superpose(prm, dev(R), t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"])
    Vu, Ou = ctx.superpose(prm, dev(R), t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"])
    torch.cuda.synchronize()
    assert float((Vw - Vu).abs().max()) < 1e-5 * float(Vu.abs().max())
    assert float((Ow - Ou).abs().max()) < 1e-5 * float(Ou.abs().max())


def test_wall_full_size_sampled(ctx, gbi):
    """The N = 10^4 trap cloud lifted above the wall (lowest centre at 2a), FP32, against
    the oracle's sums for sampled spheres."""
    c = workloads.config3()
    R = c["R"].copy()
    R[:, 2] += 2.0 * c["a"] - R[:, 2].min()
    N = len(R)
    prm_o = dict(a=c["a"], eta=c["eta"], k=c["k"], vs=c["vs"], s0=c["s0"], d0=0.0)
    inp = dynamics.trap_inputs(R, c["p"], prm_o, 2)
    prm = gbi.params(a=c["a"], eta=c["eta"], trunc=2, precision=1)
    t = {k: dev(v) for k, v in inp.items()}
    V, O = ctx.wall_superpose(prm, dev(R), t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"])
    torch.cuda.synchronize()
    tg = np.random.default_rng(9).choice(N, size=3, replace=False)
    Vo, Oo = wall.wall_superpose(R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"], c["a"], c["eta"],
                                 targets=tg)
    Vg, Og = V.cpu().numpy()[tg], O.cpu().numpy()[tg]
    assert np.abs(Vg - Vo).max() / np.linalg.norm(Vo, axis=1).max() < 1e-5
    assert np.abs(Og - Oo).max() / np.linalg.norm(Oo, axis=1).max() < 1e-5
