"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
textbook limits, exact Stokes solutions, an independent library (scipy's
spherical harmonics) or brute-force quadrature of the defining integrals.
"""
import math

import numpy as np
import pytest

from oracle import dynamics, galerkin, quadrature, taylor, tensors

ETA = 0.7
A = 1.3


# ---------------------------------------------------------------- derivatives

def test_taylor_closed_forms():
    rho = np.array([[0.3, -1.2, 2.0], [1.0, 2.0, 3.0], [-4.0, 0.5, 0.1]])
    r = np.linalg.norm(rho, axis=1)
    ix = taylor.mono_index(6)
    d1 = taylor.derivatives(rho, -1.0, 6)
    dr = taylor.derivatives(rho, 1.0, 6)
    e = np.eye(3, dtype=int)
    for i in range(3):
        np.testing.assert_allclose(d1[:, ix[tuple(e[i])]], -rho[:, i] / r ** 3, rtol=1e-13)
        np.testing.assert_allclose(dr[:, ix[tuple(e[i])]], rho[:, i] / r, rtol=1e-13)
        for j in range(3):
            n = tuple(e[i] + e[j])
            np.testing.assert_allclose(d1[:, ix[n]], (3 * rho[:, i] * rho[:, j] - (i == j) * r ** 2) / r ** 5,
                                       rtol=1e-12, atol=1e-15)
            np.testing.assert_allclose(dr[:, ix[n]], ((i == j) - rho[:, i] * rho[:, j] / r ** 2) / r,
                                       rtol=1e-12, atol=1e-15)
    # harmonicity of 1/r and biharmonicity of r, at every order available
    lap = [tuple(2 * e[i]) for i in range(3)]
    for n in taylor.monomials(4):
        s1 = sum(d1[:, ix[tuple(np.add(n, l))]] for l in lap)
        np.testing.assert_allclose(s1, 0.0, atol=1e-9 * np.abs(d1[:, ix[n]]).max() + 1e-12)
    for n in taylor.monomials(2):
        s = sum(dr[:, ix[tuple(np.add(np.add(n, l1), l2))]] for l1 in lap for l2 in lap)
        assert np.abs(s).max() < 1e-10


def test_taylor_finite_difference():
    rho = np.array([[0.7, -1.1, 1.9]])
    ix = taylor.mono_index(4)
    h = 1e-3
    for nu in (-1.0, 1.0):
        d = taylor.derivatives(rho, nu, 4)
        # d^3/dx dy dz by central differences of the third order mixed derivative
        f = lambda x: np.linalg.norm(x) ** nu
        fd = 0.0
        for sx in (-1, 1):
            for sy in (-1, 1):
                for sz in (-1, 1):
                    fd += sx * sy * sz * f(rho[0] + h * np.array([sx, sy, sz]))
        fd /= 8 * h ** 3
        assert abs(fd - d[0, ix[(1, 1, 1)]]) < 1e-5 * max(1.0, abs(fd))


# ---------------------------------------------------------------- harmonics

def test_stf_basis_matches_scipy_real_harmonics():
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(3)
    n = rng.normal(size=(50, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    theta = np.arccos(n[:, 2])
    phi = np.arctan2(n[:, 1], n[:, 0])
    for k in range(1, 6):
        U = tensors.stf_basis(k)
        Nk = math.sqrt(4 * math.pi * math.factorial(k) / tensors.dfact(2 * k + 1))
        flat = U.reshape(2 * k + 1, -1)
        np.testing.assert_allclose(flat @ flat.T, np.eye(2 * k + 1), atol=1e-12)
        for j, mu in enumerate(range(-k, k + 1)):
            m = abs(mu)
            Yc = sph_harm_y(k, m, theta, phi)           # includes (-1)^m
            if mu == 0:
                ref = Yc.real
            elif mu > 0:
                ref = math.sqrt(2) * (-1) ** m * Yc.real
            else:
                ref = math.sqrt(2) * (-1) ** m * Yc.imag
            val = np.array([np.tensordot(U[j], tensors.outer_power(v, k).reshape((3,) * k), axes=k)
                            for v in n])
            np.testing.assert_allclose(val, Nk * ref, atol=1e-11)


def test_tsh_definition_and_orthogonality():
    """Y^(l) = (-1)^l r^(l+1) grad^(l) (1/r) and the orthogonality relation (Sec. III)."""
    rng = np.random.default_rng(4)
    nvec = rng.normal(size=3)
    nvec /= np.linalg.norm(nvec)
    ix = taylor.mono_index(4)
    D = taylor.derivatives(nvec[None], -1.0, 4)[0]
    for l in range(1, 5):
        Y = tensors.tsh(l, nvec)
        for t in np.ndindex(Y.shape):
            m = [0, 0, 0]
            for i in t:
                m[i] += 1
            assert abs(Y[t] - (-1) ** l * D[ix[tuple(m)]]) < 1e-12
    pts, wts = galerkin.sphere_rule(10, 22)
    for l in range(0, 4):
        for lp in range(0, 4):
            Ys = np.array([np.ravel(tensors.tsh(l, p)) for p in pts])
            Yp = np.array([np.ravel(tensors.tsh(lp, p)) for p in pts])
            M = np.einsum("k,ka,kb->ab", wts, Ys, Yp) / (4 * np.pi)
            if l != lp:
                assert np.abs(M).max() < 1e-12
            else:
                ref = math.factorial(l) * tensors.dfact(2 * l - 1) / (2 * l + 1) * tensors.stf_projector(l)
                np.testing.assert_allclose(M, ref, atol=1e-12)


def test_embedding_coefficients_and_rigid_modes():
    """The sigma embeddings reproduce the paper's l = 3, 4 coefficients and the rigid modes."""
    rng = np.random.default_rng(5)
    for L, c1, c2 in ((3, -2 / 3, 3 / 5), (4, -3 / 4, 6 / 7)):
        T1 = tensors.unpack_stf(rng.normal(size=2 * L - 1), L - 1)
        T2 = tensors.unpack_stf(rng.normal(size=2 * L - 3), L - 2)
        E1 = tensors.embed(L, 1, T1)
        E2 = tensors.embed(L, 2, T2)
        X1 = np.tensordot(tensors.LEVI, T1, axes=([2], [0]))
        X2 = np.multiply.outer(np.eye(3), T2)
        np.testing.assert_allclose(E1, c1 * tensors._project_tail(X1), atol=1e-14)
        np.testing.assert_allclose(E2, c2 * tensors._project_tail(X2), atol=1e-14)
        # delta contraction recovers the trace part exactly at L = 3; at L = 4 the printed
        # coefficient 6/7 makes it 6/5 T (reading R3: the embedding coefficients are kept)
        ratio = 1.0 if L == 3 else 6.0 / 5.0
        np.testing.assert_allclose(np.trace(E2, axis1=0, axis2=1), ratio * T2, atol=1e-12)
    # rigid rotation v = Omega x rho has V^(2) = (3/4 pi a^2) int v rhohat dS whose sigma=1
    # part is V^(21) = 2 a Omega, which is what galerkin.lower_velocity inverts
    pts, wts = galerkin.sphere_rule(8, 16)
    Om = np.array([0.3, -0.7, 0.2])
    v = np.cross(Om, A * pts)
    V2 = 3 / (4 * np.pi) * np.einsum("k,ki,ka->ia", wts, v, pts)
    np.testing.assert_allclose(V2, tensors.embed(2, 1, 2 * A * Om), atol=1e-13)
    # a traction with torque T: F^(2) = int f rhohat dS, sigma=1 part F^(21) = T / a
    Tq = np.array([0.1, 0.5, -0.4])
    f = 3 / (8 * np.pi * A ** 4) * np.cross(Tq, A * pts)
    torque = np.einsum("k,ki->i", wts * A ** 2, np.cross(A * pts, f))
    np.testing.assert_allclose(torque, Tq, atol=1e-13)
    F2 = np.einsum("k,ki,ka->ia", wts * A ** 2, f, pts)
    np.testing.assert_allclose(F2, tensors.embed(2, 1, Tq / A), atol=1e-13)


# ---------------------------------------------------------------- self elements

def _g_by_mode(trunc, a):
    MB = tensors.ModeBasis(trunc)
    S = galerkin.self_matrix(trunc, a)
    assert np.abs(S - np.diag(np.diag(S))).max() < 1e-10 / a
    g = np.diag(S)
    out = {}
    for mi, (name, L, s) in enumerate(MB.modes):
        vals = g[MB.mode_of == mi]
        assert np.ptp(vals) < 1e-10 / a
        out[name] = vals[0]
    return out


def test_self_scalars_against_one_body_laws():
    """8 pi eta V^(ls) = -g Q^(ls) for an isolated sphere (Sec. IV, Eq.
    single_sphere_traction_velocity_relations), so g = -8 pi eta V/Q per mode."""
    g = _g_by_mode(4, A)
    a = A
    assert abs(g["1s"] - 4 / (3 * a)) < 1e-12      # Stokes drag F = 6 pi eta a V
    assert abs(g["2a"] - 2 / a) < 1e-12            # rotational drag T = 8 pi eta a^3 Omega
    assert abs(g["2s"] - 6 / (5 * a)) < 1e-12      # S = -20/3 pi eta a^3 s
    assert abs(g["3s"] - 48 / (7 * a)) < 1e-12     # Gamma = -7/6 pi eta a^5 gamma
    assert abs(g["3t"] - 4 / a) < 1e-12            # D = -2 pi eta a^5 d
    # toroidal (sigma = 1) modes: the exact exterior/interior Stokes solutions with a
    # tangential surface velocity of degree l give a single-layer density
    # q = -(2l+1) eta v / a, hence g = 2 l! (2l-1)!! / a (l = Y degree = L - 1)
    for name, l in (("2a", 1), ("3a", 2), ("4a", 3)):
        assert abs(g[name] - 2 * math.factorial(l) * tensors.dfact(2 * l - 1) / a) < 1e-9


def test_self_scalars_against_the_papers_coefficient_table():
    """The sigma = 0 single-layer entries of the paper's table of C_lsigma
    (tests/golden/one_body_coefficients.txt) give the self scalars of those modes."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "one_body_coefficients.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 2
    g = _g_by_mode(3, A)
    for name, mode, num, den, power in rows:
        l = int(name[1])
        C = float(num) / float(den) * math.pi * ETA * A ** int(power)
        assert abs(g[mode] - 8 * math.pi * ETA * A ** (2 * l - 2) / C) < 1e-12 * g[mode], name


def test_self_elements_from_exterior_flow():
    """Self elements equal the Galerkin projection of the exterior flow formula (App. B)
    evaluated on the surface, an independent route to Eq. single_layer_yl_matrix_element."""
    S1 = galerkin.self_matrix(3, A)
    S2 = quadrature.self_block_from_flow(A, 3)
    np.testing.assert_allclose(S1, S2, atol=1e-11)


# ---------------------------------------------------------------- pair elements

@pytest.mark.parametrize("rho", [[1.3 * 3.0, -0.4, 0.9], [0.2, -3.3 * 1.3, 2.2]])
def test_pair_blocks_against_double_surface_quadrature(rho):
    rho = np.array(rho)
    B = galerkin.pair_blocks(rho, A, 3)[0]
    Bq = quadrature.pair_block_bruteforce(rho, A, 3, nt=20, nphi=40)
    np.testing.assert_allclose(B, Bq, atol=1e-11 * np.abs(B).max())


def test_pair_blocks_l4_against_quadrature():
    rho = np.array([2.9, 2.1, -1.4])
    B = galerkin.pair_blocks(rho, 1.0, 4)[0]
    Bq = quadrature.pair_block_bruteforce(rho, 1.0, 4, nt=16, nphi=32)
    np.testing.assert_allclose(B, Bq, atol=1e-10 * np.abs(B).max())


def test_pair_symmetry():
    rng = np.random.default_rng(8)
    rho = rng.normal(size=(5, 3)) * 3
    B = galerkin.pair_blocks(rho, A, 4)
    Bm = galerkin.pair_blocks(-rho, A, 4)
    np.testing.assert_allclose(B, np.transpose(Bm, (0, 2, 1)), atol=1e-13 * np.abs(B).max())


def test_rpy_and_rotlet_blocks():
    """1s-1s is the Rotne-Prager-Yamakawa tensor; 2a-1s is the rotlet (F x rho)/rho^3."""
    rho = np.array([2.5, -1.0, 3.0])
    r = np.linalg.norm(rho)
    n = rho / r
    B = galerkin.pair_blocks(rho, A, 2)[0]
    P = np.array([1, 2, 0])          # packed index -> Cartesian axis
    rpy = (np.eye(3) + np.outer(n, n)) / r + 2 * A * A / 3 * (np.eye(3) - 3 * np.outer(n, n)) / r ** 3
    np.testing.assert_allclose(B[:3, :3], rpy[np.ix_(P, P)], atol=1e-14)
    # Omega_n = (F_m x rho)/(8 pi eta rho^3) for a force F_m
    MB = tensors.ModeBasis(2)
    F = np.array([0.3, 0.8, -0.5])
    xF = galerkin.lower_trial(F[None], np.zeros((1, 3)), A, MB)[0]
    xV = -(B[3:6, :3] @ xF[:3]) / (8 * np.pi * ETA)
    _, Om = galerkin.lower_velocity(np.concatenate([np.zeros(3), xV])[None], np.zeros((1, 3)),
                                    np.zeros((1, 3)), A, MB)
    np.testing.assert_allclose(Om[0], np.cross(F, rho) / (8 * np.pi * ETA * r ** 3), atol=1e-15)


# ---------------------------------------------------------------- whole system

def test_single_sphere_laws():
    R = np.zeros((1, 3))
    F = np.array([[0.2, -0.1, 0.5]])
    Tq = np.array([[0.3, 0.4, -0.2]])
    Va = np.array([[0.01, 0.02, 0.03]])
    Oa = np.array([[0.1, 0.0, -0.05]])
    VH = np.random.default_rng(0).normal(size=(1, 25))
    V, Om, QH = galerkin.solve(R, Va, Oa, VH, F, Tq, A, ETA, 3)
    np.testing.assert_allclose(V, Va + F / (6 * np.pi * ETA * A), atol=1e-15)
    np.testing.assert_allclose(Om, Oa + Tq / (8 * np.pi * ETA * A ** 3), atol=1e-15)


def test_squirmer_stresslet():
    """Squirmer: V^(20) = -3/5 B2 (pp - I/3) (Sec. V) gives the classical stresslet
    S = a Q^(20) = 4 pi eta a^2 B2 (pp - I/3) (Lighthill/Blake)."""
    B2 = 0.3
    p = np.array([0.0, 0.6, 0.8])
    P2 = np.outer(p, p) - np.eye(3) / 3
    VH = np.zeros((1, 8))
    VH[0, :5] = tensors.pack_stf(-0.6 * B2 * P2)
    _, _, QH = galerkin.solve(np.zeros((1, 3)), np.zeros((1, 3)), np.zeros((1, 3)), VH,
                              np.zeros((1, 3)), np.zeros((1, 3)), A, ETA, 2)
    S = A * tensors.unpack_stf(QH[0, :5], 2)
    np.testing.assert_allclose(S, 4 * np.pi * ETA * A ** 2 * B2 * P2, atol=1e-14)


def test_strain_mode_exterior_flow_is_single_layer_of_Q():
    """Reading R1: the exterior flow of a sphere whose surface moves with v = E.x
    (classical solution u = 5a^3/2 (xEx)x/r^5 + a^5 [E.x/r^5 - 5/2 (xEx)x/r^7])
    equals the single-layer flow of the density whose 2s coefficient is the oracle's
    one-body Q^(20) -- so the flow is carried by Q, not by the bare traction moment."""
    rng = np.random.default_rng(11)
    E = rng.normal(size=(3, 3))
    E = (E + E.T) / 2
    E -= np.trace(E) / 3 * np.eye(3)
    VH = np.zeros((1, 8))
    VH[0, :5] = tensors.pack_stf(A * E)                 # V^(20) = a s with s = E
    Q20 = tensors.unpack_stf(galerkin.one_body_QH(VH, A, ETA, 2)[0, :5], 2)
    pts, wts = galerkin.sphere_rule(20, 40)
    q = 3 / (4 * np.pi * A ** 2) * pts @ Q20.T           # (2l+1)/(4 pi a^2) Q^(2) . Y^(1)
    for x in rng.normal(size=(4, 3)) * 3:
        x = x / np.linalg.norm(x) * (A * 2.2)
        r = np.linalg.norm(x)
        xEx = x @ E @ x
        exact = 2.5 * A ** 3 * xEx * x / r ** 5 + A ** 5 * (E @ x / r ** 5 - 2.5 * xEx * x / r ** 7)
        G = quadrature.stokeslet(x[None] - A * pts)
        u = -np.einsum("k,kij,kj->i", wts * A ** 2, G, q) / (8 * np.pi * ETA)
        np.testing.assert_allclose(u, exact, atol=1e-12)


def test_two_sphere_far_field_mobility():
    """Two equal spheres, force on one along the line of centres: the self mobility
    is 1 - 15/4 (a/r)^4 + O((a/r)^6) (classical two-sphere expansion)."""
    coefs = []
    for r in (16.0, 32.0):
        R = np.array([[0, 0, 0], [r * A, 0, 0]])
        F = np.array([[1.0, 0, 0], [0, 0, 0]])
        V, _, _ = galerkin.solve(R, np.zeros((2, 3)), np.zeros((2, 3)), np.zeros((2, 25)), F,
                                 np.zeros((2, 3)), A, ETA, 3)
        coefs.append((V[0, 0] * 6 * np.pi * ETA * A - 1.0) * r ** 4)
    extrap = coefs[1] + (coefs[1] - coefs[0]) / 3.0       # O(r^-2) relative remainder
    assert abs(extrap + 15.0 / 4.0) < 2e-3


def test_spd_and_grand_mobility():
    import workloads
    s = workloads.small_cloud(6, 1)
    R = s["R"] * A
    N = len(R)
    for trunc in (2, 3):
        MB = tensors.ModeBasis(trunc)
        Afull = galerkin.assemble(R, A, trunc).reshape(N, MB.d, N, MB.d)
        AHH = Afull[:, MB.nL:, :, MB.nL:].reshape(N * MB.h, -1)
        np.testing.assert_allclose(AHH, AHH.T, atol=1e-14)
        np.linalg.cholesky(AHH)
    # passive grand mobility from unit forces / torques: symmetric positive definite
    M = np.zeros((6 * N, 6 * N))
    for col in range(6 * N):
        F = np.zeros((N, 3))
        Tq = np.zeros((N, 3))
        (F if col < 3 * N else Tq).reshape(-1)[col % (3 * N)] = 1.0
        V, Om, _ = galerkin.solve(R, np.zeros((N, 3)), np.zeros((N, 3)), np.zeros((N, 8)), F, Tq,
                                  A, ETA, 2)
        M[:, col] = np.concatenate([V.reshape(-1), Om.reshape(-1)])
    np.testing.assert_allclose(M, M.T, atol=1e-12 * np.abs(M).max())
    assert np.linalg.eigvalsh((M + M.T) / 2).min() > 0


def _rot(seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def test_invariance_translation_rotation_permutation():
    import workloads
    s = workloads.small_cloud(5, 2)
    R, p = s["R"] * A, s["p"]
    prm = dict(a=A, eta=ETA, k=0.02, vs=0.1, s0=0.05, d0=0.03)
    V, Om = dynamics.velocities(R, p, prm, 3, False)
    V2, Om2 = dynamics.velocities(R + np.array([5.0, -2.0, 1.0]), p, dict(prm, k=0.0), 3, False)
    V3, Om3 = dynamics.velocities(R, p, dict(prm, k=0.0), 3, False)
    np.testing.assert_allclose(V2, V3, atol=1e-14)
    np.testing.assert_allclose(Om2, Om3, atol=1e-14)
    Q = _rot(3)
    V4, Om4 = dynamics.velocities(R @ Q.T, p @ Q.T, prm, 3, False)
    np.testing.assert_allclose(V4, V @ Q.T, atol=1e-13)
    np.testing.assert_allclose(Om4, Om @ Q.T, atol=1e-13)
    perm = np.array([3, 0, 4, 1, 2])
    V5, Om5 = dynamics.velocities(R[perm], p[perm], prm, 3, False)
    np.testing.assert_allclose(V5, V[perm], atol=1e-14)
    np.testing.assert_allclose(Om5, Om[perm], atol=1e-14)


@pytest.mark.parametrize("case", ["pair", "triangle"])
def test_truncation_convergence(case):
    """Two and three active spheres in the trap at centre distances 2.05a, 2.5a, 3a, 4a:
    the change of (V, Omega) from one truncation to the next, l <= 2, 3, 4, 5, 6, decreases
    monotonically, and the paper's minimal truncation (every mode of rank <= 4, 47
    components per sphere, Sec. IV) is closer to l <= 6 than l <= 3 is."""
    prm = dict(a=A, eta=ETA, k=0.01, vs=0.1, s0=0.05, d0=0.02)
    for r in (2.05, 2.5, 3.0, 4.0):
        if case == "pair":
            R = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]]) * A
            p = np.array([[0.0, 0.6, 0.8], [1.0, 0.0, 0.0]])
        else:
            R = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0], [r / 2, r * math.sqrt(3) / 2, 0.0]]) * A
            p = np.array([[0.0, 0.6, 0.8], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
        out = {tr: np.concatenate(dynamics.velocities(R, p, prm, tr, False), axis=1).ravel()
               for tr in (2, 3, 4, 5, 6, tensors.MINIMAL)}
        steps = [np.linalg.norm(out[b] - out[a]) for a, b in ((2, 3), (3, 4), (4, 5), (5, 6))]
        assert all(y < x for x, y in zip(steps, steps[1:])), (r, steps)
        assert np.linalg.norm(out[tensors.MINIMAL] - out[6]) < np.linalg.norm(out[3] - out[6])
    assert tensors.ModeBasis(tensors.MINIMAL).d == 47


def test_superposition_is_dilute_limit():
    """Full solve minus superposition decays faster than the pair interaction itself."""
    p = np.array([[0, 0, 1.0], [0.6, 0, 0.8]])
    prm = dict(a=A, eta=ETA, k=0.05, vs=0.1, s0=0.05, d0=0.0)
    rel = []
    for sep in (4.0, 8.0, 16.0):
        R = np.array([[0, 0, 0], [sep * A, 0.3, 0.1]])
        Vf, _ = dynamics.velocities(R, p, prm, 2, False)
        Vs, _ = dynamics.velocities(R, p, prm, 2, True)
        V1, _ = dynamics.velocities(R[:1], p[:1], prm, 2, True)
        rel.append(np.linalg.norm(Vf[0] - Vs[0]) / np.linalg.norm(Vs[0] - V1[0]))
    assert rel[2] < rel[1] < rel[0]
    assert rel[2] < 0.05


# ---------------------------------------------------------------- trap dynamics

def test_trap_single_particle_relaxation_and_fixed_point():
    prm = dict(a=A, eta=ETA, k=0.02, vs=0.0, s0=0.0, d0=0.0)
    R0 = np.array([[3.0, -1.0, 2.0]])
    p0 = np.array([[0.0, 0.0, 1.0]])
    dt, n = 0.5, 20
    R, _ = dynamics.trajectory(R0, p0, prm, 2, dt, n, superposition=True)
    tau1 = 6 * np.pi * ETA * A / prm["k"]
    np.testing.assert_allclose(R, R0 * (1 - dt / tau1) ** n, rtol=1e-12)
    # active particle: fixed point at R* = 6 pi eta v_s a / k along p
    prm = dict(prm, vs=0.1, s0=0.05)
    Rstar = 6 * np.pi * ETA * prm["vs"] * A / prm["k"]
    V, Om = dynamics.velocities(np.array([[0, 0, Rstar]]), p0, prm, 2, True)
    assert np.abs(V).max() < 1e-15 and np.abs(Om).max() < 1e-15


def test_trap_opposite_pair_does_not_rotate():
    """Two squirmers at diametrically opposite points of the R* sphere, pointing
    outwards: Omega = 0 identically (Sec. V, two-particle discussion)."""
    prm = dict(a=A, eta=ETA, k=0.01, vs=0.1, s0=0.05, d0=0.0)
    Rstar = 6 * np.pi * ETA * prm["vs"] * A / prm["k"]
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    R = np.array([Rstar * u, -Rstar * u])
    p = np.array([u, -u])
    for sup in (True, False):
        _, Om = dynamics.velocities(R, p, prm, 2, sup)
        assert np.abs(Om).max() < 1e-16


# ---------------------------------------------------------------- active modes and kinematics

def _curl_and_laplacian(u, x, h=1e-2):
    """Fourth-order central differences of a closed-form field u at x."""
    e = np.eye(3)
    J = np.zeros((3, 3))                                  # J[i, j] = d u_i / d x_j
    lap = np.zeros(3)
    for j in range(3):
        f = [u(x + k * h * e[j]) for k in (-2, -1, 0, 1, 2)]
        J[:, j] = (f[0] - 8 * f[1] + 8 * f[3] - f[4]) / (12 * h)
        lap += (-f[0] + 16 * f[1] - 30 * f[2] + 16 * f[3] - f[4]) / (12 * h * h)
    curl = np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])
    return curl, lap


@pytest.mark.parametrize("trunc", [2, 3])
def test_active_strain_mode_drives_passive_partner(trunc):
    """``active_modes`` with s0 != 0 only: V^(2s) = s0 (pp - I/3) = a E (Sec. V trap
    parametrisation; Sec. III, v = V^(2).Y^(1) on the surface).  The exterior flow of
    that sphere is the classical strain solution u_E; a passive, force- and torque-free
    partner in the superposition approximation moves with the Faxen laws
    V = (1 + a^2/6 lap) u_E and Omega = curl(u_E)/2 at its centre (Sec. IV, first
    terms of the superposition mobility).  A wrong sign, slot or scale of s0 fails."""
    s0 = 0.07
    p = np.array([[0.36, -0.48, 0.8]])
    E = s0 * (np.outer(p[0], p[0]) - np.eye(3) / 3) / A

    def u_E(x):
        r = np.linalg.norm(x)
        xEx = x @ E @ x
        return 2.5 * A ** 3 * xEx * x / r ** 5 + A ** 5 * (E @ x / r ** 5 - 2.5 * xEx * x / r ** 7)

    MB = tensors.ModeBasis(trunc)
    VH = np.zeros((2, MB.h))
    VH[:1] = galerkin.active_modes(p, s0, 0.0, trunc)
    z = np.zeros((2, 3))
    for x2 in (np.array([5.0, 2.0, -1.5]) * A, np.array([-1.0, 3.0, 4.0]) * A):
        R = np.array([np.zeros(3), x2])
        V, Om = galerkin.superpose(R, z, z, VH, z, z, A, ETA, trunc)
        curl, lap = _curl_and_laplacian(u_E, x2)
        np.testing.assert_allclose(V[1], u_E(x2) + A ** 2 / 6 * lap, rtol=1e-7, atol=1e-12)
        np.testing.assert_allclose(Om[1], curl / 2, rtol=1e-7, atol=1e-12)
        np.testing.assert_allclose(V[0], 0.0, atol=1e-16)
        np.testing.assert_allclose(Om[0], 0.0, atol=1e-16)


@pytest.mark.parametrize("trunc", [2, 3])
def test_active_dipole_mode_drives_passive_partner(trunc):
    """``active_modes`` with d0 != 0 only: V^(3t) = d0 p, the trace part of V^(3) with the
    embedding coefficient 3/5 (Sec. III, Eq. irred_velocity_coefficients_inverse), so the
    surface velocity (1/3!!2!) V^(3):Y^(2) is v = (3 nn - I).d/10 (Sec. III expansion of v).
    Its exterior flow is the potential dipole u = (d0/10)(a/r)^3 (3 (p.r^) r^ - p), harmonic,
    so a passive partner moves with exactly u and does not rotate."""
    d0 = -0.09
    p = np.array([[0.0, 0.6, -0.8]])
    MB = tensors.ModeBasis(trunc)
    VH = np.zeros((2, MB.h))
    VH[:1] = galerkin.active_modes(p, 0.0, d0, trunc)
    z = np.zeros((2, 3))
    for x2 in (np.array([4.0, -2.0, 1.0]) * A, np.array([0.5, 1.0, -6.0]) * A):
        R = np.array([np.zeros(3), x2])
        V, Om = galerkin.superpose(R, z, z, VH, z, z, A, ETA, trunc)
        r = np.linalg.norm(x2)
        n = x2 / r
        u = d0 / 10 * (A / r) ** 3 * (3 * (p[0] @ n) * n - p[0])
        np.testing.assert_allclose(V[1], u, rtol=1e-12, atol=1e-16)
        np.testing.assert_allclose(Om[1], 0.0, atol=1e-16)


def test_euler_turns_orientation_about_the_torque():
    """One sphere under a force F and a torque T perpendicular to p: V = F/(6 pi eta a),
    Omega = T/(8 pi eta a^3) (Stokes laws, Sec. IV).  Forward Euler on dp/dt = Omega x p
    (Sec. II kinematics) followed by renormalisation turns p about T, in the right-handed
    sense, by exactly atan(dt |Omega|) per step, and moves R by dt V."""
    F = np.array([[0.2, -0.1, 0.05]])
    T = np.array([[0.0, 0.0, 0.9]])
    R = np.array([[1.0, 2.0, -3.0]])
    p = np.array([[0.8, 0.6, 0.0]])
    dt = 0.3
    z = np.zeros((1, 3))
    for _ in range(5):
        V, Om, _ = galerkin.solve(R, z, z, np.zeros((1, 8)), F, T, A, ETA, 2)
        Rn, pn = dynamics.euler(R, p, V, Om, dt)
        w = T[0, 2] / (8 * np.pi * ETA * A ** 3)
        ang = math.atan(dt * w)
        np.testing.assert_allclose(Rn, R + dt * F / (6 * np.pi * ETA * A), rtol=1e-14)
        np.testing.assert_allclose(np.linalg.norm(pn[0]), 1.0, rtol=1e-15)
        # counter-clockwise about +z: p_new = Rz(ang) p
        c, s = math.cos(ang), math.sin(ang)
        expect = np.array([c * p[0, 0] - s * p[0, 1], s * p[0, 0] + c * p[0, 1], 0.0])
        np.testing.assert_allclose(pn[0], expect, atol=1e-14)
        assert np.cross(p[0], pn[0])[2] > 0
        R, p = Rn, pn


# ---------------------------------------------------------------- flow field

def _exterior_points(R0, rng, n, rmin, rmax):
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return R0 + d * rng.uniform(rmin, rmax, size=(n, 1)) * A


def test_flow_of_translating_and_rotating_sphere():
    """One sphere under a force F and a torque T: the flow of the Galerkin representation
    is the exact exterior Stokes solution, F.[(1/r + a^2/3r^3) I + (1/r^3 - a^2/r^5) rho rho]
    / (8 pi eta) (translation) plus T x rho / (8 pi eta r^3) (rotation)."""
    from oracle import flow
    rng = np.random.default_rng(21)
    R0 = np.array([[0.4, -1.0, 2.0]])
    F = np.array([[0.3, -0.7, 0.2]])
    T = np.array([[-0.2, 0.5, 0.9]])
    z = np.zeros((1, 3))
    _, _, QH = galerkin.solve(R0, z, z, np.zeros((1, 25)), F, T, A, ETA, 3)
    X = _exterior_points(R0[0], rng, 12, 2.0, 6.0)
    U = flow.flow(X, R0, flow.internal_coefficients(F, T, QH, A, 3), A, ETA, 3)
    rho = X - R0
    r = np.linalg.norm(rho, axis=1)[:, None]
    exact = (F * (1 / r + A ** 2 / (3 * r ** 3)) + rho * np.sum(rho * F, axis=1, keepdims=True)
             * (1 / r ** 3 - A ** 2 / r ** 5)) / (8 * np.pi * ETA) + np.cross(T, rho) / (8 * np.pi * ETA * r ** 3)
    np.testing.assert_allclose(U, exact, rtol=1e-11, atol=1e-14)


def test_flow_of_strain_and_dipole_modes():
    """One force-free sphere with only the strain mode V^(2s) = a E, then only the dipole
    mode V^(3t) = d: its flow is the classical strain solution, then the potential dipole
    (d/10)(a/r)^3 (3 (d.r^) r^ - d) (both derived from the surface velocity v = V^(l+1).Y^(l)
    / (l!(2l-1)!!) of Sec. III)."""
    from oracle import flow
    rng = np.random.default_rng(22)
    R0 = np.zeros((1, 3))
    z = np.zeros((1, 3))
    E = rng.normal(size=(3, 3))
    E = (E + E.T) / 2
    E -= np.trace(E) / 3 * np.eye(3)
    d = rng.normal(size=3)
    for which in ("strain", "dipole"):
        VH = np.zeros((1, 8))
        if which == "strain":
            VH[0, :5] = tensors.pack_stf(A * E)
        else:
            VH[0, 5:8] = galerkin.vec_to_packed(d)
        _, _, QH = galerkin.solve(R0, z, z, VH, z, z, A, ETA, 2)
        X = _exterior_points(R0[0], rng, 10, 1.6, 5.0)
        U = flow.flow(X, R0, flow.internal_coefficients(z, z, QH, A, 2), A, ETA, 2)
        r = np.linalg.norm(X, axis=1)[:, None]
        if which == "strain":
            xEx = np.einsum("mi,ij,mj->m", X, E, X)[:, None]
            exact = 2.5 * A ** 3 * xEx * X / r ** 5 + A ** 5 * (X @ E.T / r ** 5 - 2.5 * xEx * X / r ** 7)
        else:
            n = X / r
            exact = (A / r) ** 3 * (3 * (n @ d)[:, None] * n - d) / 10
        np.testing.assert_allclose(U, exact, rtol=1e-10, atol=1e-14)


# ---------------------------------------------------------------- squirmer

def test_squirmer_modes_from_the_slip():
    """Squirmer slip v^a = (nn - I).[B1 p + B2 (pp - I/3).n] (Sec. V): its tensorial-harmonic
    coefficients give the printed V^a = 2 B1 p / 3 and V^(20) = -3/5 B2 (pp - I/3), no
    rotation, the potential dipole V^(32) = 10/3 B1 p and the degenerate octupole
    V^(42) = 7 B2 (pp - I/3) in the oracle's embedding (the slip's l = 2 and l = 3 parts,
    (B1/3) Y^(2).p and (B2/15)(pp - I/3):Y^(3)), and nothing else; the expansion
    sum_l V^(l+1).Y^(l) / (l!(2l-1)!!) rebuilds the slip."""
    from oracle.tensors import dfact, tsh
    rng = np.random.default_rng(31)
    p = rng.normal(size=3)
    p /= np.linalg.norm(p)
    B1, B2 = 0.21, -0.37
    S = np.outer(p, p) - np.eye(3) / 3
    Va, Oa, VH = dynamics.squirmer_modes(p, B1, B2, 3)
    np.testing.assert_allclose(Va, 2 * B1 / 3 * p, atol=1e-14)
    np.testing.assert_allclose(Oa, 0.0, atol=1e-14)
    np.testing.assert_allclose(VH[0:5], tensors.pack_stf(-0.6 * B2 * S), atol=1e-14)
    np.testing.assert_allclose(VH[5:8], galerkin.vec_to_packed(10 / 3 * B1 * p), atol=1e-14)
    np.testing.assert_allclose(VH[8:20], 0.0, atol=1e-14)                 # 3a, 3s
    np.testing.assert_allclose(VH[20:25], tensors.pack_stf(7 * B2 * S), atol=1e-13)
    # rebuild the slip from the reducible coefficients of the truncation (l <= 3)
    MB = tensors.ModeBasis(3)
    y = np.concatenate([galerkin.vec_to_packed(-Va), np.zeros(3), VH])
    n = rng.normal(size=(6, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    v = np.zeros((6, 3))
    for L in (1, 2, 3, 4):
        l = L - 1
        T = sum(y[i] * MB.scale[i] * e for i, e in enumerate(MB.vectors) if MB.rank[i] == L)
        for k in range(6):
            Y = tsh(l, n[k])
            v[k] += (np.tensordot(T, Y, axes=l) if l > 0 else T * Y) / (math.factorial(l) * dfact(2 * l - 1))
    np.testing.assert_allclose(v, dynamics.squirmer_slip(p, B1, B2, n), atol=1e-13)
