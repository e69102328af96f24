"""Flow field at points in the fluid (gbi_flow) against the oracle.

The oracle evaluates the Galerkin representation by surface quadrature of the single
layer of every sphere's flow-coefficient density (oracle/flow.py, pinned against exact
exterior Stokes solutions); the GPU sums the multipole form of the same single layer
(the 1s row of the pair operator for a target of radius zero).  Also: the surface
average of the flow just outside a sphere equals that sphere's velocity from the solve
(the 1s Galerkin condition), points inside a sphere are flagged, and the N = 1024
suspension is checked at sampled points.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle import dynamics, flow, galerkin

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


def _points_outside(R, a, rng, n, dmin):
    lo, hi = R.min(axis=0) - 4 * a, R.max(axis=0) + 4 * a
    out = []
    while len(out) < n:
        x = rng.uniform(lo, hi)
        if np.linalg.norm(R - x, axis=1).min() >= dmin * a:
            out.append(x)
    return np.array(out)


@pytest.mark.parametrize("trunc", [2, 3, 4, 5, 40])
@pytest.mark.parametrize("precision", [0, 1])
def test_flow_matches_oracle_quadrature(ctx, gbi, trunc, precision):
    if trunc in (5, 40) and precision == 1:
        pytest.skip("l <= 5 and the minimal truncation run in FP64 only")
    s = workloads.small_cloud(4, 60 + trunc, phi=0.1)
    R, p = s["R"], s["p"]
    prm_o = dict(a=s["a"], eta=s["eta"], k=s["k"], vs=s["vs"], s0=s["s0"], d0=0.03)
    inp = dynamics.trap_inputs(R, p, prm_o, trunc)
    inp["Te"] = np.random.default_rng(trunc).normal(size=(len(R), 3)) * 0.02
    inp["VH"] = inp["VH"] + np.random.default_rng(10 + trunc).normal(size=inp["VH"].shape) * 0.01
    _, _, QH = galerkin.solve(R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"], s["a"], s["eta"], trunc)
    X = _points_outside(R, s["a"], np.random.default_rng(7), 30, 2.0)
    ref = flow.flow(X, R, flow.internal_coefficients(inp["Fe"], inp["Te"], QH, s["a"], trunc), s["a"], s["eta"],
                    trunc)
    prm = gbi.params(a=s["a"], eta=s["eta"], trunc=trunc, precision=precision)
    U, n_in = ctx.flow(prm, dev(R), dev(inp["Fe"]), dev(inp["Te"]), dev(QH), dev(X))
    torch.cuda.synchronize()
    assert n_in == 0
    err = np.abs(U.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < (1e-10 if precision == 0 else 1e-5), err


def test_flow_surface_average_is_the_sphere_velocity(ctx, gbi):
    """Just outside sphere n the flow is the surface velocity; its average over S_n is the
    translational velocity V_n of the solve (the 1s row of the Galerkin condition), with
    every other sphere's and sphere n's own single layer included."""
    s = workloads.small_cloud(6, 61, phi=0.1)
    R, p = s["R"], s["p"]
    trunc = 3
    prm_o = dict(a=s["a"], eta=s["eta"], k=s["k"], vs=0.0, s0=0.0, d0=0.0)
    inp = dynamics.trap_inputs(R, p, prm_o, trunc)          # passive spheres in the trap
    prm = gbi.params(a=s["a"], eta=s["eta"], trunc=trunc, precision=0, rtol=1e-12)
    t = {k: dev(v) for k, v in inp.items()}
    V, Om, QH, info, _ = ctx.solve(prm, dev(R), t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"])
    pts, wts = galerkin.sphere_rule(16, 32)
    for n in (0, 3):
        X = R[n] + s["a"] * (1 + 1e-9) * pts
        U, n_in = ctx.flow(prm, dev(R), t["Fe"], t["Te"], QH, dev(X))
        torch.cuda.synchronize()
        assert n_in == 0
        avg = (wts[:, None] * U.cpu().numpy()).sum(axis=0) / wts.sum()
        Vn = V.cpu().numpy()[n]
        assert np.abs(avg - Vn).max() < 1e-7 * np.abs(V.cpu().numpy()).max()


def test_flow_flags_points_inside_spheres(ctx, gbi):
    R = np.array([[0.0, 0.0, 0.0], [5.0, 0.0, 0.0]])
    z = np.zeros((2, 3))
    F = np.array([[0.1, 0.0, 0.0], [0.0, 0.0, 0.0]])
    prm = gbi.params(a=1.0, eta=1.0, trunc=2, precision=1)
    X = np.array([[0.3, 0.1, 0.0], [2.5, 0.0, 0.0], [5.0, 0.9, 0.0], [0.0, 3.0, 0.0]])
    U, n_in = ctx.flow(prm, dev(R), dev(F), dev(z), dev(np.zeros((2, 8))), dev(X))
    torch.cuda.synchronize()
    U = U.cpu().numpy()
    assert n_in == 2
    assert np.all(np.isnan(U[[0, 2]])) and np.all(np.isfinite(U[[1, 3]]))


def test_flow_full_size_sampled(ctx, gbi):
    """N = 1024, l <= 3: the GPU's solve (double-float refinement) and flow field at
    sampled points between the spheres, against the oracle's quadrature of the same Q^H."""
    c = workloads.config2()
    R, p = c["R"], c["p"]
    N = len(R)
    inp = ctx.trap_inputs(N, 3, c["k"], c["vs"], c["s0"], c["d0"], dev(R), dev(p))
    prm = gbi.params(a=c["a"], eta=c["eta"], trunc=3, precision=2, rtol=1e-10)
    V, Om, QH, info, _ = ctx.solve(prm, dev(R), inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
    X = _points_outside(R, c["a"], np.random.default_rng(8), 40, 2.0)
    X = X[np.linalg.norm(X, axis=1) < 20][:6]   # among the spheres
    assert len(X) == 6
    prm1 = gbi.params(a=c["a"], eta=c["eta"], trunc=3, precision=1)
    U, n_in = ctx.flow(prm1, dev(R), inp["Fe"], inp["Te"], QH, dev(X))
    torch.cuda.synchronize()
    xi = flow.internal_coefficients(inp["Fe"].cpu().numpy(), inp["Te"].cpu().numpy(), QH.cpu().numpy(), c["a"], 3)
    ref = flow.flow(X, R, xi, c["a"], c["eta"], 3)
    assert n_in == 0
    assert np.abs(U.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-5
