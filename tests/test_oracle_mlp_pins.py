"""Pins of the learned near-field oracle (oracle/mlp.py) against what mathematics fixes.

* loss gradient against central finite differences (FP64, one- and two-pair spheres);
* the pair frame is orthonormal and right-handed, p_n lies in its x-z half plane,
  and the degenerate branches still give a frame;
* rotating the whole configuration leaves the features unchanged and rotates the
  predicted velocities with it (the frame is attached to the pair);
* Adam's first two steps against their closed forms;
* bfloat16 round-to-nearest-even on values whose rounding is known by hand;
* a network with zero weights outputs its last bias.
"""
import numpy as np
import pytest

from oracle import mlp


def random_theta(rng, scale=0.3):
    return rng.normal(scale=scale, size=mlp.NPARAM)


def random_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def three_body(rng):
    R = np.array([[0.0, 0.0, 0.0], [2.6, 0.4, -0.3], [0.7, 2.9, 0.5]])
    return R, unit(rng, 3)


def test_finite_difference_gradient():
    rng = np.random.default_rng(0)
    theta = random_theta(rng, 0.2)
    R, p = three_body(rng)
    tg, sr = mlp.pair_list(R, 1.0)
    assert len(tg) == 6
    F, FR = mlp.features_for_pairs(R, p, 1.0, tg, sr)
    labels = rng.normal(size=(3, 6))
    loss, g = mlp.loss_and_grad(theta, F, FR, tg, labels)
    idx = rng.choice(mlp.NPARAM, size=60, replace=False)
    # make sure every block of the layout is probed
    starts = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])[:-1]
    idx = np.concatenate([idx, starts, starts + 1])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = mlp.loss_and_grad(tp, F, FR, tg, labels)
        lm, _ = mlp.loss_and_grad(tm, F, FR, tg, labels)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_frame_invariants_and_degenerate_branches():
    rng = np.random.default_rng(1)
    for _ in range(50):
        rho = rng.normal(size=3) * 3
        pn, pm = unit(rng, 2)
        fr = mlp.pair_frame(rho, pn, pm)
        np.testing.assert_allclose(fr @ fr.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(fr) == pytest.approx(1.0, abs=1e-14)
        np.testing.assert_allclose(fr[2], rho / np.linalg.norm(rho), atol=1e-15)
        assert abs(pn @ fr[1]) < 1e-14 and pn @ fr[0] >= 0
    rho = np.array([0.0, 0.0, 3.0])
    fr = mlp.pair_frame(rho, np.array([0.0, 0.0, 1.0]), np.array([0.6, 0.8, 0.0]))
    np.testing.assert_allclose(fr[0], [0.6, 0.8, 0.0], atol=1e-15)      # falls back to p_m
    fr = mlp.pair_frame(rho, np.array([0.0, 0.0, -1.0]), np.array([0.0, 0.0, 1.0]))
    np.testing.assert_allclose(fr[0], [1.0, 0.0, 0.0], atol=1e-15)      # falls back to the x axis
    np.testing.assert_allclose(fr @ fr.T, np.eye(3), atol=1e-15)


def test_features_invariant_and_prediction_equivariant_under_rotation():
    rng = np.random.default_rng(2)
    theta = random_theta(rng)
    R, p = three_body(rng)
    tg, sr = mlp.pair_list(R, 1.0)
    F, FR = mlp.features_for_pairs(R, p, 1.0, tg, sr)
    out = mlp.predict(theta, F, FR, tg, 3)
    Q = random_rotation(rng)
    R2, p2 = (R + [5.0, -1.0, 2.0]) @ Q.T, p @ Q.T
    F2, FR2 = mlp.features_for_pairs(R2, p2, 1.0, tg, sr)
    np.testing.assert_allclose(F2, F, atol=1e-12)
    out2 = mlp.predict(theta, F2, FR2, tg, 3)
    np.testing.assert_allclose(out2[:, :3], out[:, :3] @ Q.T, atol=1e-12)
    np.testing.assert_allclose(out2[:, 3:], out[:, 3:] @ Q.T, atol=1e-12)


def test_feature_values_of_a_simple_pair():
    rho = np.array([0.0, 0.0, 3.0])
    pn = np.array([1.0, 0.0, 0.0])
    pm = np.array([0.0, 1.0, 0.0])
    f, fr = mlp.pair_features(rho, pn, pm, 1.0)
    np.testing.assert_allclose(f, [2 / 3, 8 / 27, 1.0, 0.0, 0.0, 1.0, 0.0, 1.0, 0.0], atol=1e-15)


def test_pair_list_cutoff_and_systems():
    R = np.array([[0.0, 0, 0], [3.9, 0, 0], [8.0, 0, 0], [0.0, 0, 0], [0.0, 4.1, 0]])
    tg, sr = mlp.pair_list(R, 1.0, offsets=[0, 3, 5])
    assert list(zip(tg, sr)) == [(0, 1), (1, 0)]


def test_adam_closed_form_first_steps():
    rng = np.random.default_rng(3)
    th = rng.normal(size=7)
    g1, g2 = rng.normal(size=7), rng.normal(size=7)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    t1, m, v = mlp.adam_step(th, g1, np.zeros(7), np.zeros(7), 1, lr)
    np.testing.assert_allclose(t1, th - lr * g1 / (np.abs(g1) + eps), rtol=0, atol=1e-15)
    t2, _, _ = mlp.adam_step(t1, g2, m, v, 2, lr)
    mh = (b1 * (1 - b1) * g1 + (1 - b1) * g2) / (1 - b1 ** 2)
    vh = (b2 * (1 - b2) * g1 ** 2 + (1 - b2) * g2 ** 2) / (1 - b2 ** 2)
    np.testing.assert_allclose(t2, t1 - lr * mh / (np.sqrt(vh) + eps), rtol=0, atol=1e-15)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2.0 ** -9, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -8 + 2.0 ** -9, -2.5, 0.0, 3.0e38])
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -7, -2.5, 0.0, 2.9908e38])
    got = mlp.bf16_round(x)
    np.testing.assert_allclose(got[:6], want[:6], rtol=0, atol=0)
    assert abs(got[6] - 3.0e38) / 3.0e38 < 2 ** -8


def test_zero_network_outputs_last_bias():
    theta = np.zeros(mlp.NPARAM)
    P = mlp.unflatten(theta)
    P["b4"][:] = [1, 2, 3, 4, 5, 6]
    F = np.random.default_rng(4).normal(size=(5, mlp.NIN))
    o, _ = mlp.forward(theta, F)
    np.testing.assert_allclose(o, np.tile([1, 2, 3, 4, 5, 6], (5, 1)))


# ------------------------------------------------------------------ strain-mode head

def _pack_uniaxial(u):
    from oracle import tensors
    return tensors.pack_stf(np.outer(u, u) - np.eye(3) / 3)


def test_strain_head_takes_frame_tensors_to_the_lab():
    """A uniaxial tensor along a frame axis (pair-frame coordinates e_k e_k - I/3) becomes
    e_k e_k - I/3 in the lab, for every axis of random frames; the map is orthogonal
    on the five tensor outputs and leaves the spare output alone."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        rho = rng.normal(size=3) * 3
        pn, pm = unit(rng, 2)
        fr = mlp.pair_frame(rho, pn, pm)
        for k in range(3):
            o = np.zeros((1, 6))
            o[0, :5] = _pack_uniaxial(np.eye(3)[k])
            o[0, 5] = 0.7
            lab = mlp.rotate_out(o, fr[None], head=1)
            np.testing.assert_allclose(lab[0, :5], _pack_uniaxial(fr[k]), atol=1e-14)
            assert lab[0, 5] == 0.7
        M = mlp.head_matrices(fr[None], head=1)[0]
        np.testing.assert_allclose(M[:5, :5] @ M[:5, :5].T, np.eye(5), atol=1e-13)
        assert np.all(M[5, :5] == 0) and np.all(M[:5, 5] == 0) and M[5, 5] == 1.0


def test_strain_head_prediction_equivariant_under_rotation():
    """Rotating the configuration rotates every predicted Q^(2s) tensor with it:
    S -> Q S Q^T (the frame is attached to the pair)."""
    from oracle import tensors
    rng = np.random.default_rng(12)
    theta = random_theta(rng)
    R, p = three_body(rng)
    tg, sr = mlp.pair_list(R, 1.0)
    F, FR = mlp.features_for_pairs(R, p, 1.0, tg, sr)
    out = mlp.predict(theta, F, FR, tg, 3, head=1)
    Q = random_rotation(rng)
    F2, FR2 = mlp.features_for_pairs((R + [1.0, 2.0, -3.0]) @ Q.T, p @ Q.T, 1.0, tg, sr)
    out2 = mlp.predict(theta, F2, FR2, tg, 3, head=1)
    for n in range(3):
        S = tensors.unpack_stf(out[n, :5], 2)
        np.testing.assert_allclose(out2[n, :5], tensors.pack_stf(Q @ S @ Q.T), atol=1e-12)
    np.testing.assert_allclose(out2[:, 5], out[:, 5], atol=1e-12)


def test_finite_difference_gradient_strain_head():
    rng = np.random.default_rng(13)
    theta = random_theta(rng, 0.2)
    R, p = three_body(rng)
    tg, sr = mlp.pair_list(R, 1.0)
    F, FR = mlp.features_for_pairs(R, p, 1.0, tg, sr)
    labels = rng.normal(size=(3, 6))
    loss, g = mlp.loss_and_grad(theta, F, FR, tg, labels, head=1)
    starts = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])[:-1]
    idx = np.concatenate([rng.choice(mlp.NPARAM, size=40, replace=False), starts, starts + 1])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = mlp.loss_and_grad(tp, F, FR, tg, labels, head=1)
        lm, _ = mlp.loss_and_grad(tm, F, FR, tg, labels, head=1)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_strain_labels_vanish_when_spheres_separate():
    """The strain-mode label is the solve's Q^(2s) minus the one-body one: it decays with
    the separation of two spheres (as (a/r)^3 from the leading strain-strain coupling,
    Sec. III) and is exactly zero for a single sphere."""
    from oracle import dynamics, galerkin
    prm = dict(a=1.0, eta=1.0, k=0.0, vs=0.1, s0=0.05, d0=0.0)
    p = np.array([[0.0, 0.6, 0.8], [1.0, 0.0, 0.0]])
    mags = []
    for r in (3.0, 6.0, 12.0):
        R = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
        inp = dynamics.trap_inputs(R, p, prm, 4)
        _, _, QH = galerkin.solve(R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"], 1.0, 1.0, 4)
        lab = mlp.labels_qstrain(QH, galerkin.one_body_QH(inp["VH"], 1.0, 1.0, 4), 0.05, 1.0)
        assert np.all(lab[:, 5] == 0.0)
        mags.append(np.abs(lab[:, :5]).max())
    assert mags[0] > mags[1] > mags[2] > 0
    assert 4.0 < mags[1] / mags[2] < 16.0          # between (a/r)^2 and (a/r)^4 at large r
    R1 = np.zeros((1, 3))
    inp = dynamics.trap_inputs(R1, p[:1], prm, 4)
    _, _, QH = galerkin.solve(R1, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"], 1.0, 1.0, 4)
    lab = mlp.labels_qstrain(QH, galerkin.one_body_QH(inp["VH"], 1.0, 1.0, 4), 0.05, 1.0)
    assert np.abs(lab).max() < 1e-12
