"""Learned near-field correction on the GPU against the FP64 oracle (oracle/mlp.py).

* neighbour lists: the exact set of pairs closer than rcut a (integer work: bit-exact);
* features: FP32 against FP64, 2e-5 absolute;
* tensor-core inference: the oracle multiplies the same bf16-rounded weights and layer
  inputs in FP64; a rounding decision of an activation can still differ by one bf16
  step (2^-8 relative), so outputs agree to 1e-2 of their largest magnitude;
* training gradient (FP32 CUDA cores) against the oracle's backpropagation: 2e-2 in
  relative 2-norm (same bf16 argument); Adam step: FP32 against FP64, 1e-5;
* labels: the batched l <= 4 solve per system against single solves, and the batched
  superposition against the single-system one;
* the trained network reduces the error of the superposition approximation against
  the plain l <= 4 solve, on held-out systems and on a dense suspension.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gbi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1411_0278_gb300 as g
    g.lib()
    return g


@pytest.fixture()
def ctx(gbi):
    c = gbi.Context(0)
    yield c
    c.close()


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def brute_pairs(R, rc, offsets=None):
    """Plain definition, vectorised: (dx dx + dy dy) + dz dz < rc^2, sorted by (n, m)."""
    N = len(R)
    offsets = [0, N] if offsets is None else offsets
    tg, sr = [], []
    for s in range(len(offsets) - 1):
        lo, hi = offsets[s], offsets[s + 1]
        X = R[lo:hi]
        d = X[:, None, :] - X[None, :, :]
        d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
        np.fill_diagonal(d2, np.inf)
        n, m = np.nonzero(d2 < rc * rc)
        tg.append(n + lo)
        sr.append(m + lo)
    return np.concatenate(tg), np.concatenate(sr)


@pytest.mark.parametrize("N,phi,cells", [(300, 0.1, False), (6000, 0.1, True), (5000, 0.02, True)])
def test_pairs_exact_set(ctx, gbi, N, phi, cells):
    s = workloads.suspension(N, phi, 2.05, workloads.SEED_BASE + 500 + N)
    R = s["R"] + np.array([1.0e3, -2.0e3, 5.0])
    tg, sr = ctx.pairs(dev(R), 1.0, 4.0)
    bt, bs = brute_pairs(R, 4.0)
    assert len(bt) > N
    np.testing.assert_array_equal(tg.cpu().numpy(), bt)
    np.testing.assert_array_equal(sr.cpu().numpy(), bs)


def test_pairs_batched_systems(ctx, gbi):
    d = workloads.nearfield_systems(40, 60, k=1)
    tg, sr = ctx.pairs(dev(d["R"]), 1.0, 4.0, d["offsets"])
    bt, bs = brute_pairs(d["R"], 4.0, d["offsets"])
    np.testing.assert_array_equal(tg.cpu().numpy(), bt)
    np.testing.assert_array_equal(sr.cpu().numpy(), bs)
    t2, s2 = omlp.pair_list(d["R"][:50], 1.0, [o for o in d["offsets"] if o <= 50])
    np.testing.assert_array_equal(tg.cpu().numpy()[:len(t2)], t2)


def _random_pairs(P, seed):
    rng = np.random.default_rng(seed)
    R = rng.uniform(-20, 20, size=(2 * P, 3))
    R[1::2] = R[0::2] + workloads.unit_vectors(P, rng) * rng.uniform(2.0, 4.0, size=(P, 1))
    p = workloads.unit_vectors(2 * P, rng)
    if P > 2:
        p[4] = (R[4] - R[5]) / np.linalg.norm(R[4] - R[5])      # p_n along the axis: p_m branch
    tg = np.arange(0, 2 * P, 2)
    sr = tg + 1
    return R, p, tg, sr


def test_features_match_oracle(ctx, gbi):
    R, p, tg, sr = _random_pairs(700, 3)
    F, FR = ctx.mlp_features(dev(R), dev(p), dev(tg, torch.int32), dev(sr, torch.int32), 1.0)
    Fo, FRo = omlp.features_for_pairs(R, p, 1.0, tg, sr)
    np.testing.assert_allclose(F.cpu().numpy(), Fo, atol=2e-5, rtol=0)
    np.testing.assert_allclose(FR.cpu().numpy().reshape(-1, 3, 3), FRo, atol=2e-5, rtol=0)


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("P", [1, 63, 64, 127, 128, 1000])
def test_tensor_core_forward_matches_oracle(ctx, gbi, P, engine):
    from paper_1411_0278_gb300 import nearfield
    th = nearfield.init_theta(7)
    th[omlp.NPARAM - 6:] = [0.1, -0.2, 0.3, 0.0, 0.05, -0.05]
    ctx.mlp_set(th, 4.0)
    ctx.mlp_set_engine(engine)
    R, p, tg, sr = _random_pairs(P, 5 + P)
    Fo, FRo = omlp.features_for_pairs(R, p, 1.0, tg, sr)
    Fd = dev(Fo, torch.float32)
    out = ctx.mlp_forward(Fd).cpu().numpy()
    ref, _ = omlp.forward(th.astype(np.float64), Fo.astype(np.float32).astype(np.float64), bf16=True)
    scale = np.abs(ref).max()
    assert np.abs(out - ref).max() <= 1e-2 * scale
    if P >= 64:
        # the bulk of the outputs much closer, and no systematic offset
        assert np.median(np.abs(out - ref)) <= 3e-3 * scale
        assert np.abs(np.mean(out - ref, axis=0)).max() <= 1e-3 * scale
    lab = ctx.mlp_forward(Fd, dev(FRo.reshape(-1, 9), torch.float32)).cpu().numpy()
    np.testing.assert_allclose(lab, omlp.rotate_out(ref, FRo), atol=1e-2 * scale, rtol=0)
    ctx.mlp_status()


def test_engines_agree(ctx, gbi):
    """Both inference engines multiply the same bf16 values; only FP32 summation order and
    an occasional bf16 rounding of an activation differ."""
    from paper_1411_0278_gb300 import nearfield
    ctx.mlp_set(nearfield.init_theta(9), 1.0)
    R, p, tg, sr = _random_pairs(5000, 12)
    F, FR = ctx.mlp_features(dev(R), dev(p), dev(tg, torch.int32), dev(sr, torch.int32), 1.0)
    ctx.mlp_set_engine(0)
    a = ctx.mlp_forward(F).cpu().numpy()
    ctx.mlp_set_engine(1)
    b = ctx.mlp_forward(F).cpu().numpy()
    ctx.mlp_status()
    assert np.abs(a - b).max() <= 1e-2 * np.abs(a).max()
    assert np.median(np.abs(a - b)) <= 1e-4 * np.abs(a).max()


@pytest.mark.parametrize("engine", [0, 1])
def test_training_gradient_matches_oracle(ctx, gbi, engine):
    """Both training engines against the oracle's gradient: engine 0 (FP32 CUDA cores) and
    engine 1 (tcgen05: the inference forward, bf16 GEMM operands in the backward)."""
    from paper_1411_0278_gb300 import nearfield
    d = workloads.nearfield_systems(30, 50, k=2)
    th = nearfield.init_theta(11)
    ctx.mlp_set(th, 2.0)
    ctx.mlp_set_engine(engine)
    rng = np.random.default_rng(4)
    labels = rng.normal(size=(len(d["R"]), 6))
    loss, g = ctx.mlp_loss_grad(dev(d["R"]), dev(d["p"]), 1.0, dev(labels), d["offsets"])
    tg, sr = omlp.pair_list(d["R"], 1.0, d["offsets"])
    F, FR = omlp.features_for_pairs(d["R"], d["p"], 1.0, tg, sr)
    lo, go = omlp.loss_and_grad(th.astype(np.float64), F, FR, tg, labels, bf16=True)
    ctx.mlp_status()
    assert abs(loss - lo) <= 2e-3 * lo
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - go) <= 2e-2 * np.linalg.norm(go)
    for name, shp in omlp.SHAPES:      # every block of the layout carries gradient
        k0 = sum(int(np.prod(s)) for n_, s in omlp.SHAPES[:[n for n, _ in omlp.SHAPES].index(name)])
        blk = slice(k0, k0 + int(np.prod(shp)))
        assert np.linalg.norm(g[blk] - go[blk]) <= 5e-2 * np.linalg.norm(go[blk]), name


def test_training_gradient_many_tiles(ctx, gbi):
    """~7e4 pairs (several 128-pair tiles per block of the tensor-core backward, whose
    weight gradients accumulate in tensor memory across them): both engines against the
    oracle, and against each other."""
    from paper_1411_0278_gb300 import nearfield
    d = workloads.nearfield_systems(3000, 12000, k=5)
    th = nearfield.init_theta(13)
    ctx.mlp_set(th, 2.0)
    labels = np.random.default_rng(6).normal(size=(len(d["R"]), 6))
    tg, sr = omlp.pair_list(d["R"], 1.0, d["offsets"])
    assert len(tg) > 128 * 2 * 152
    F, FR = omlp.features_for_pairs(d["R"], d["p"], 1.0, tg, sr)
    lo, go = omlp.loss_and_grad(th.astype(np.float64), F, FR, tg, labels, bf16=True)
    gs = []
    for engine in (0, 1):
        ctx.mlp_set_engine(engine)
        loss, g = ctx.mlp_loss_grad(dev(d["R"]), dev(d["p"]), 1.0, dev(labels), d["offsets"])
        ctx.mlp_status()
        g = g.cpu().numpy().astype(np.float64)
        assert abs(loss - lo) <= 2e-3 * lo, engine
        assert np.linalg.norm(g - go) <= 2e-2 * np.linalg.norm(go), engine
        gs.append(g)
    assert np.linalg.norm(gs[1] - gs[0]) <= 2e-2 * np.linalg.norm(gs[0])


def test_adam_matches_oracle(ctx, gbi):
    from paper_1411_0278_gb300 import nearfield
    th = nearfield.init_theta(3)
    ctx.mlp_set(th, 1.0)
    rng = np.random.default_rng(8)
    g1, g2 = rng.normal(size=omlp.NPARAM), rng.normal(size=omlp.NPARAM)
    ctx.mlp_adam(dev(g1, torch.float32), 1e-3)
    ctx.mlp_adam(dev(g2, torch.float32), 5e-4)
    got, sig = ctx.mlp_get()
    # both inference engines follow the updated weights
    R, p, tg, sr = _random_pairs(300, 21)
    F = dev(omlp.features_for_pairs(R, p, 1.0, tg, sr)[0], torch.float32)
    outs = []
    for engine in (0, 1):
        ctx.mlp_set_engine(engine)
        outs.append(ctx.mlp_forward(F).cpu().numpy())
    ctx.mlp_status()
    ref, _ = omlp.forward(got.astype(np.float64), F.cpu().numpy().astype(np.float64), bf16=True)
    for o in outs:
        assert np.abs(o - ref).max() <= 1e-2 * np.abs(ref).max()
    assert sig == 1.0
    t = th.astype(np.float64)
    m = np.zeros_like(t)
    v = np.zeros_like(t)
    t, m, v = omlp.adam_step(t, g1.astype(np.float32).astype(np.float64), m, v, 1, 1e-3)
    t, m, v = omlp.adam_step(t, g2.astype(np.float32).astype(np.float64), m, v, 2, 5e-4)
    np.testing.assert_allclose(got, t, atol=1e-6, rtol=1e-5)


@pytest.mark.parametrize("engine", [0, 1])
def test_correct_adds_scaled_sums(ctx, gbi, engine):
    from paper_1411_0278_gb300 import nearfield
    s = workloads.suspension(400, 0.1, 2.05, workloads.SEED_BASE + 77)
    th = nearfield.init_theta(5)
    ctx.mlp_set(th, 8.0)
    ctx.mlp_set_engine(engine)
    R, p = dev(s["R"]), dev(s["p"])
    V0 = torch.randn(400, 3, dtype=torch.float64, device="cuda")
    O0 = torch.randn(400, 3, dtype=torch.float64, device="cuda")
    V, O = V0.clone(), O0.clone()
    npairs = ctx.mlp_correct(R, p, 1.0, 0.05, V, O)
    tg, sr = omlp.pair_list(s["R"], 1.0)
    assert npairs == len(tg)
    F, FR = omlp.features_for_pairs(s["R"], s["p"], 1.0, tg, sr)
    pred = omlp.predict(th.astype(np.float64), F, FR, tg, 400, bf16=True) * (0.05 / 8.0)
    got = np.concatenate([(V - V0).cpu().numpy(), (O - O0).cpu().numpy()], axis=1)
    assert np.abs(got - pred).max() <= 1e-2 * np.abs(pred).max()


def test_batched_labels_match_single_system_calls(ctx, gbi):
    """Label inputs: batched l <= 4 solve and l <= 2 superposition per system = single calls."""
    from paper_1411_0278_gb300 import nearfield
    d = workloads.nearfield_systems(3, 4, k=3)
    R, p = dev(d["R"]), dev(d["p"])
    Vx, Ox, Vs, Os, _ = nearfield.exact_and_superposition(ctx, R, p, d["offsets"], 1.0, d["eta"], d["vs"], d["s0"])
    prm4 = gbi.params(a=1.0, eta=d["eta"], trunc=4, precision=0, rtol=1e-12, restart=60)
    prm2 = gbi.params(a=1.0, eta=d["eta"], trunc=2, precision=0)
    for s in range(len(d["offsets"]) - 1):
        lo, hi = d["offsets"][s], d["offsets"][s + 1]
        Rs, ps = R[lo:hi].contiguous(), p[lo:hi].contiguous()
        i4 = ctx.trap_inputs(hi - lo, 4, 0.0, d["vs"], d["s0"], 0.0, Rs, ps)
        V, O, _, _, _ = ctx.solve(prm4, Rs, i4["Va"], i4["Oa"], i4["VH"], i4["Fe"], i4["Te"])
        i2 = ctx.trap_inputs(hi - lo, 2, 0.0, d["vs"], d["s0"], 0.0, Rs, ps)
        V2, O2 = ctx.superpose(prm2, Rs, i2["Va"], i2["Oa"], i2["VH"], i2["Fe"], i2["Te"])
        torch.cuda.synchronize()
        sc = float((V - i4["Va"]).abs().max())
        assert float((Vx[lo:hi] - V).abs().max()) <= 1e-8 * sc
        assert float((Ox[lo:hi] - O).abs().max()) <= 1e-8 * float(O.abs().max())
        assert float((Vs[lo:hi] - V2).abs().max()) <= 1e-10 * sc
        assert float((Os[lo:hi] - O2).abs().max()) <= 1e-10 * float(O2.abs().max())


def test_trained_network_beats_superposition(ctx, gbi):
    """Train on 2- and 3-sphere systems; on held-out systems and on a dense suspension the
    network must cut the error of the superposition approximation against the l <= 4 solve."""
    from paper_1411_0278_gb300 import nearfield
    tr = workloads.nearfield_systems(3000, 3000, k=10)
    te = workloads.nearfield_systems(300, 300, k=11)
    a, eta, vs, s0 = 1.0, tr["eta"], tr["vs"], tr["s0"]
    dtr = nearfield.make_dataset(ctx, dev(tr["R"]), dev(tr["p"]), tr["offsets"], a, eta, vs, s0)
    hist = nearfield.train(ctx, dtr, epochs=40, batch_systems=256, lr0=3e-3, lr1=1e-4, seed=1)
    assert hist[-1] < 0.5 * hist[0]
    dte = nearfield.make_dataset(ctx, dev(te["R"]), dev(te["p"]), te["offsets"], a, eta, vs, s0,
                                 sigma=dtr["sigma"])
    ev = nearfield.evaluate(ctx, dte)
    assert ev["with_network"]["V"] < 0.5 * ev["superposition"]["V"], ev
    assert ev["with_network"]["Omega"] < 0.5 * ev["superposition"]["Omega"], ev
    # a dense suspension (volume fraction 0.1, 2.05a exclusion) against the plain solve
    s = workloads.suspension(300, 0.1, 2.05, workloads.SEED_BASE + 5300)
    dsus = nearfield.make_dataset(ctx, dev(s["R"]), dev(s["p"]), [0, 300], a, eta, vs, s0, sigma=dtr["sigma"])
    ev2 = nearfield.evaluate(ctx, dsus)
    assert ev2["with_network"]["V"] < ev2["superposition"]["V"], ev2


def test_nearfield_edge_cases(ctx, gbi):
    """Empty input, a single sphere, spheres farther apart than the cut-off, and a batch
    whose systems have no pairs: no pairs, nothing added."""
    from paper_1411_0278_gb300 import nearfield
    ctx.mlp_set(nearfield.init_theta(2), 1.0)
    R0 = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    assert ctx.mlp_correct(R0, R0, 1.0, 0.05, R0, R0) == 0
    tg, sr = ctx.pairs(R0, 1.0, 4.0)
    assert tg.numel() == 0
    for R in ([[0.0, 0.0, 0.0]], [[0.0, 0.0, 0.0], [4.0, 0.0, 0.0], [0.0, 9.0, 0.0]]):
        Rd = dev(R)
        p = dev(workloads.unit_vectors(len(R), np.random.default_rng(0)))
        V = torch.ones((len(R), 3), dtype=torch.float64, device="cuda")
        O = torch.ones_like(V)
        assert ctx.mlp_correct(Rd, p, 1.0, 0.05, V, O) == 0
        assert float((V - 1).abs().max()) == 0.0 and float((O - 1).abs().max()) == 0.0
    # two systems of two spheres each, pairs only inside each system
    R = dev([[0.0, 0, 0], [3.0, 0, 0], [0.5, 0, 0], [10.0, 0, 0]])
    tg, sr = ctx.pairs(R, 1.0, 4.0, [0, 2, 4])
    assert list(zip(tg.cpu().tolist(), sr.cpu().tolist())) == [(0, 1), (1, 0)]
    with pytest.raises(gbi.GbiError):
        ctx.pairs(R, 1.0, 4.0, [0, 2, 3])          # offsets must end at N


# ------------------------------------------------------------------ strain-mode head

@pytest.mark.parametrize("engine", [0, 1])
def test_strain_head_forward_matches_oracle(ctx, gbi, engine):
    """Head 1: the pair-frame outputs as before, the lab-frame ones as packed tensors
    sum_kl S'_kl e_k e_l (the oracle's map, pinned against uniaxial tensors)."""
    from paper_1411_0278_gb300 import nearfield
    th = nearfield.init_theta(17)
    th[omlp.NPARAM - 6:] = [0.1, -0.2, 0.3, 0.05, -0.05, 0.02]
    ctx.mlp_set(th, 4.0)
    ctx.mlp_set_head(1)
    ctx.mlp_set_engine(engine)
    R, p, tg, sr = _random_pairs(333, 40)
    Fo, FRo = omlp.features_for_pairs(R, p, 1.0, tg, sr)
    ref, _ = omlp.forward(th.astype(np.float64), Fo.astype(np.float32).astype(np.float64), bf16=True)
    lab = ctx.mlp_forward(dev(Fo, torch.float32), dev(FRo.reshape(-1, 9), torch.float32)).cpu().numpy()
    ctx.mlp_status()
    want = omlp.rotate_out(ref, FRo, head=1)
    assert np.abs(lab - want).max() <= 1e-2 * np.abs(want).max()


@pytest.mark.parametrize("engine", [0, 1])
def test_strain_head_gradient_matches_oracle(ctx, gbi, engine):
    from paper_1411_0278_gb300 import nearfield
    d = workloads.nearfield_systems(30, 50, k=12)
    th = nearfield.init_theta(19)
    ctx.mlp_set(th, 2.0)
    ctx.mlp_set_head(1)
    ctx.mlp_set_engine(engine)
    labels = np.random.default_rng(5).normal(size=(len(d["R"]), 6))
    loss, g = ctx.mlp_loss_grad(dev(d["R"]), dev(d["p"]), 1.0, dev(labels), d["offsets"])
    tg, sr = omlp.pair_list(d["R"], 1.0, d["offsets"])
    F, FR = omlp.features_for_pairs(d["R"], d["p"], 1.0, tg, sr)
    lo, go = omlp.loss_and_grad(th.astype(np.float64), F, FR, tg, labels, bf16=True, head=1)
    assert abs(loss - lo) <= 2e-3 * lo
    g = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - go) <= 2e-2 * np.linalg.norm(go)


def test_qh_onebody_matches_oracle(ctx, gbi):
    from oracle import dynamics, galerkin
    rng = np.random.default_rng(6)
    for trunc in (2, 3, 4):
        R = rng.normal(size=(9, 3)) * 5
        p = workloads.unit_vectors(9, rng)
        inp = dynamics.trap_inputs(R, p, dict(a=1.3, eta=0.7, k=0.0, vs=0.1, s0=0.05, d0=0.02), trunc)
        VH = inp["VH"] + rng.normal(size=inp["VH"].shape) * 0.01
        prm = gbi.params(a=1.3, eta=0.7, trunc=trunc, precision=0)
        got = ctx.qh_onebody(prm, dev(VH)).cpu().numpy()
        np.testing.assert_allclose(got, galerkin.one_body_QH(VH, 1.3, 0.7, trunc), rtol=1e-13, atol=0)


def test_strain_labels_match_oracle(ctx, gbi):
    """Labels of the strain head from the GPU's batched l <= 4 solve and one-body Q^H,
    against the oracle's dense solve of the same 2- and 3-sphere systems."""
    from oracle import dynamics, galerkin
    from paper_1411_0278_gb300 import nearfield
    d = workloads.nearfield_systems(3, 3, k=13)
    data = nearfield.make_dataset_qh(ctx, dev(d["R"]), dev(d["p"]), d["offsets"], 1.0, d["eta"], d["vs"], d["s0"])
    prm_o = dict(a=1.0, eta=d["eta"], k=0.0, vs=d["vs"], s0=d["s0"], d0=0.0)
    for s in range(len(d["offsets"]) - 1):
        lo, hi = d["offsets"][s], d["offsets"][s + 1]
        R, p = d["R"][lo:hi], d["p"][lo:hi]
        inp = dynamics.trap_inputs(R, p, prm_o, 4)
        _, _, QH = galerkin.solve(R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"], 1.0, d["eta"], 4)
        want = omlp.labels_qstrain(QH, galerkin.one_body_QH(inp["VH"], 1.0, d["eta"], 4), d["s0"], data["sigma"])
        got = data["labels"][lo:hi].cpu().numpy()
        assert np.abs(got - want).max() <= 1e-7 * np.abs(want).max(), s


def test_correct_qh_adds_scaled_sums(ctx, gbi):
    from paper_1411_0278_gb300 import nearfield
    s = workloads.suspension(400, 0.1, 2.05, workloads.SEED_BASE + 78)
    th = nearfield.init_theta(6)
    ctx.mlp_set(th, 8.0)
    ctx.mlp_set_head(1)
    R, p = dev(s["R"]), dev(s["p"])
    Q0 = torch.randn(400, 48, dtype=torch.float64, device="cuda")
    Q = Q0.clone()
    npairs = ctx.mlp_correct_qh(R, p, 1.0, 0.05, Q)
    tg, sr = omlp.pair_list(s["R"], 1.0)
    assert npairs == len(tg)
    F, FR = omlp.features_for_pairs(s["R"], s["p"], 1.0, tg, sr)
    pred = omlp.predict(th.astype(np.float64), F, FR, tg, 400, bf16=True, head=1) * (0.05 / 8.0)
    got = (Q - Q0).cpu().numpy()
    assert np.abs(got[:, :5] - pred[:, :5]).max() <= 1e-2 * np.abs(pred[:, :5]).max()
    assert np.all(got[:, 5:] == 0.0)
    # each correction needs its own head
    with pytest.raises(gbi.GbiError):
        ctx.mlp_correct(R, p, 1.0, 0.05, Q0[:, :3].contiguous(), Q0[:, 3:6].contiguous())
    ctx.mlp_set_head(0)
    with pytest.raises(gbi.GbiError):
        ctx.mlp_correct_qh(R, p, 1.0, 0.05, Q)


def test_warm_started_graph_solve_matches_host_sequence(gbi):
    """A repeated warm-started mixed solve on a user stream replays the solve graph (the
    guess packed ahead of it); it returns the host-driven sequence's solution."""
    from oracle import dynamics
    c = workloads.small_cloud(80, 90, phi=0.1)
    inp = dynamics.trap_inputs(c["R"], c["p"], dict(a=c["a"], eta=c["eta"], k=c["k"], vs=c["vs"], s0=c["s0"],
                                                     d0=0.0), 3)
    t = {k: dev(v) for k, v in inp.items()}
    prm = gbi.params(a=c["a"], eta=c["eta"], trunc=3, precision=2, rtol=1e-10)
    guess = torch.randn(80, gbi.h(3), dtype=torch.float64, device="cuda") * 1e-3
    host = gbi.Context(0)
    Q0 = guess.clone()
    V0, O0, Q0, i0, _ = host.solve(prm, dev(c["R"]), t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"], QH=Q0,
                                   warm_start=True)
    torch.cuda.synchronize()
    host.close()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = gbi.Context(0, stream=stream)
        for _ in range(3):
            Q1 = guess.clone()
            V1, O1, Q1, i1, _ = g.solve(prm, dev(c["R"]), t["Va"], t["Oa"], t["VH"], t["Fe"], t["Te"], QH=Q1,
                                        warm_start=True)
        stream.synchronize()
        assert g.solve_graph_replays() >= 1
        g.close()
    # both meet the tolerance; the host sequence orthogonalises with the fused kernel and the
    # graph with separate kernels (another summation order), so a refinement decision at
    # the tolerance may fall one sweep apart
    assert i1.rel_residual <= 1e-10 and i0.rel_residual <= 1e-10
    assert abs(i1.refinements - i0.refinements) <= 1 and abs(i1.iters - i0.iters) <= 4
    assert float((V1 - V0).abs().max()) <= 1e-8 * float(V0.abs().max())
    assert float((Q1 - Q0).abs().max()) <= 1e-7 * float(Q0.abs().max())


def test_trained_strain_head_improves_the_warm_start(ctx, gbi):
    """Train the strain head on 2- and 3-sphere systems; on held-out systems and a dense
    suspension the learned Q^(2s) is closer to the solve's than the one-body value, and
    the solve warm-started from the learned guess reaches the same solution."""
    from paper_1411_0278_gb300 import nearfield
    tr = workloads.nearfield_systems(2000, 2000, k=20)
    te = workloads.nearfield_systems(300, 300, k=21)
    a, eta, vs, s0 = 1.0, tr["eta"], tr["vs"], tr["s0"]
    dtr = nearfield.make_dataset_qh(ctx, dev(tr["R"]), dev(tr["p"]), tr["offsets"], a, eta, vs, s0)
    hist = nearfield.train_qh(ctx, dtr, epochs=30, batch_systems=256, lr0=3e-3, lr1=1e-4, seed=2)
    assert hist[-1] < 0.5 * hist[0]
    dte = nearfield.make_dataset_qh(ctx, dev(te["R"]), dev(te["p"]), te["offsets"], a, eta, vs, s0,
                                    sigma=dtr["sigma"])
    ev = nearfield.evaluate_qh(ctx, dte)
    assert ev["with_network"]["Q2s"] < 0.5 * ev["one_body"]["Q2s"], ev
    s = workloads.suspension(300, 0.1, 2.05, workloads.SEED_BASE + 5301)
    R, p = dev(s["R"]), dev(s["p"])
    dsus = nearfield.make_dataset_qh(ctx, R, p, [0, 300], a, eta, vs, s0, sigma=dtr["sigma"])
    ev2 = nearfield.evaluate_qh(ctx, dsus)
    assert ev2["with_network"]["Q2s"] < ev2["one_body"]["Q2s"], ev2
    prm = gbi.params(a=a, eta=eta, trunc=4, precision=2, rtol=1e-10)
    inp = ctx.trap_inputs(300, 4, 0.0, vs, s0, 0.0, R, p)
    Vz, Oz, Qz, iz, _ = ctx.solve(prm, R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
    Qg = nearfield.guess_qh(ctx, prm, R, p, inp["VH"], s0)
    Vg, Og, Qg, ig, _ = ctx.solve(prm, R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"], QH=Qg,
                                  warm_start=True)
    torch.cuda.synchronize()
    assert ig.rel_residual <= 1e-10
    assert float((Vg - Vz).abs().max()) <= 1e-8 * float((Vz - inp["Va"]).abs().max())
