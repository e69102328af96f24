"""Learned near-field correction: pair features, network, loss, gradients, Adam (FP64).

TEST INFRASTRUCTURE ONLY (see the package header): this is the slow, plain
reference the CUDA training and inference kernels are compared against.

The paper has no network.  What is learned is the difference between two of its
results for the same spheres: the Galerkin solution of the boundary-integral
equations (Sec. II, Eq. many_body_active_passive_stresses, solved at truncation
l <= 4) and the superposition approximation of Sec. IV (one-body traction
coefficients, direct pair sums only).  The model is pairwise: every ordered pair
(n, m) closer than 4a contributes a correction to the translational and angular
velocity of n, predicted in a frame attached to the pair and rotated back.

Pair frame (n the target, m the source, rho = R_n - R_m):
    e_z = rho / r;
    e_x = the part of p_n normal to e_z, normalised; if |.|^2 <= 1e-12 the part of
          p_m normal to e_z; if that is also degenerate, the coordinate axis with
          the smallest |e_z component| (first such axis) made normal to e_z;
    e_y = e_z x e_x.
Features (9):  2a/r, (2a/r)^3, d, ln d, p_n.e_z, p_n.e_x, p_m.e_x, p_m.e_y, p_m.e_z
    with d = max(r/a - 2, 0.01).
Network: tanh layers 9 -> 128 -> 128 -> 128, linear output 6 (o_0..2 the velocity,
o_3..5 the angular velocity, both in the pair frame).  The correction of n is
    dV_n = (s0 / sigma) sum_m sum_c o_c e_c,  dOmega_n = (s0 / sigma) sum_m sum_c o_(3+c) e_c,
s0 the strain amplitude of the workload and sigma the label scale of the model.

Flat parameter layout (shared with the C ABI): W1[128][9], b1[128], W2[128][128],
b2[128], W3[128][128], b3[128], W4[6][128], b4[6]  (35 078 numbers).

Second head (head = 1): the six outputs of a pair are instead o_0..4 = the packed
coordinates of a symmetric traceless tensor S' in the pair frame (the orthonormal STF
packing of tensors.pack_stf) and o_5, trained toward zero and unused.  Its lab-frame
contribution is pack(sum_kl S'_kl e_k e_l), and the per-sphere sum predicts the
correction of the strain-mode flow coefficient Q^(2s) (the first five packed components
of Q^H, Sec. III Eq. generalized_Qlsigma) beyond its one-body value
(galerkin.one_body_QH):  labels_n = sigma/s0 (Q^(2s)_solve - Q^(2s)_one-body, 0).

Loss over a set of spheres with labels L_n (6 numbers, already scaled by sigma/s0):
    loss = sum_n |P_n - L_n|^2 / (6 Ns),   P_n = sum over n's pairs of the rotated o.
Adam: Kingma & Ba (2015), bias-corrected first and second moments.

Pins: tests/test_oracle_mlp_pins.py (central finite differences of the loss,
frame invariants and rotation equivariance, Adam's closed-form first steps,
bf16 round-to-nearest-even on known values, the zero-weight network).
"""
import numpy as np

NIN, NH, NOUT = 9, 128, 6
RCUT = 4.0          # pairs with r < RCUT * a are corrected
SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("W3", (NH, NH)), ("b3", (NH,)),
          ("W4", (NOUT, NH)), ("b4", (NOUT,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(theta):
    """Flat parameter vector -> dict of arrays (views)."""
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[k:k + n].reshape(shp)
        k += n
    return out


def flatten(params):
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16_round(x):
    """Round to the nearest bfloat16 (8 significand bits), ties to even, as float64.

    Done on the float32 bit pattern: add 0x7FFF plus the lowest kept bit, clear the
    low 16 bits.  Inputs are first rounded to float32 (the GPU's master copy)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def pair_frame(rho, pn, pm):
    """Rows e_x, e_y, e_z of the pair frame (3x3) for one ordered pair."""
    r = np.sqrt(rho @ rho)
    ez = rho / r
    t = pn - (pn @ ez) * ez
    if t @ t <= 1e-12:
        t = pm - (pm @ ez) * ez
    if t @ t <= 1e-12:
        k = int(np.argmin(np.abs(ez)))
        e = np.zeros(3)
        e[k] = 1.0
        t = e - ez[k] * ez
    ex = t / np.sqrt(t @ t)
    ey = np.cross(ez, ex)
    return np.stack([ex, ey, ez])


def pair_features(rho, pn, pm, a):
    """(9 features, 3x3 frame) of the ordered pair with rho = R_n - R_m."""
    fr = pair_frame(rho, pn, pm)
    r = np.sqrt(rho @ rho)
    u = 2.0 * a / r
    d = max(r / a - 2.0, 0.01)
    ex, ey, ez = fr
    f = np.array([u, u ** 3, d, np.log(d), pn @ ez, pn @ ex, pm @ ex, pm @ ey, pm @ ez])
    return f, fr


def pair_list(R, a, offsets=None, rcut=RCUT):
    """Ordered pairs (n, m), n != m, of the same system with |R_n - R_m| < rcut a,
    sorted by n then m.  offsets: system boundaries (None = one system).  Brute force."""
    N = len(R)
    if offsets is None:
        offsets = [0, N]
    tg, sr = [], []
    for s in range(len(offsets) - 1):
        lo, hi = offsets[s], offsets[s + 1]
        for n in range(lo, hi):
            for m in range(lo, hi):
                if m == n:
                    continue
                d = R[n] - R[m]
                if (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2] < (rcut * a) ** 2:
                    tg.append(n)
                    sr.append(m)
    return np.array(tg, dtype=np.int64), np.array(sr, dtype=np.int64)


def features_for_pairs(R, p, a, tg, sr):
    F = np.zeros((len(tg), NIN))
    FR = np.zeros((len(tg), 3, 3))
    for k, (n, m) in enumerate(zip(tg, sr)):
        F[k], FR[k] = pair_features(R[n] - R[m], p[n], p[m], a)
    return F, FR


def forward(theta, F, bf16=False):
    """Network outputs o [P, 6] and the cache of the backward pass.

    bf16=True rounds the weights and every layer input to bfloat16 before the
    product (what the tensor-core inference kernel multiplies); sums stay FP64."""
    P = unflatten(theta)
    rd = bf16_round if bf16 else (lambda v: v)
    x0 = rd(F)
    z1 = x0 @ rd(P["W1"]).T + P["b1"]
    h1 = np.tanh(z1)
    z2 = rd(h1) @ rd(P["W2"]).T + P["b2"]
    h2 = np.tanh(z2)
    z3 = rd(h2) @ rd(P["W3"]).T + P["b3"]
    h3 = np.tanh(z3)
    o = rd(h3) @ rd(P["W4"]).T + P["b4"]
    return o, (x0, h1, h2, h3)


def rotate_out(o, FR, head=0):
    """Lab-frame contributions [P, 6] from pair-frame outputs: head 0, (dV, dOmega) =
    sum_c o_c e_c for each triple; head 1, pack(sum_kl S'_kl e_k e_l) with
    S' = unpack(o_0..4), and o_5 unchanged."""
    o = np.asarray(o, float)
    if head == 0:
        v = np.einsum("pc,pci->pi", o[:, :3], FR)
        w = np.einsum("pc,pci->pi", o[:, 3:], FR)
        return np.concatenate([v, w], axis=1)
    from .tensors import pack_stf, unpack_stf
    out = np.zeros_like(o)
    for k in range(len(o)):
        S = unpack_stf(o[k, :5], 2)                  # pair-frame coordinates
        out[k, :5] = pack_stf(FR[k].T @ S @ FR[k])   # sum_kl S_kl e_k e_l (rows e_k of FR)
        out[k, 5] = o[k, 5]
    return out


def head_matrices(FR, head=0):
    """The linear map of rotate_out for every pair, [P, 6, 6] (lab = M o), built by
    applying rotate_out to the unit outputs."""
    P = len(FR)
    M = np.zeros((P, NOUT, NOUT))
    for c in range(NOUT):
        e = np.zeros((P, NOUT))
        e[:, c] = 1.0
        M[:, :, c] = rotate_out(e, FR, head)
    return M


def predict(theta, F, FR, tg, Ns, bf16=False, head=0):
    """Per-sphere sums P_n [Ns, 6] (label units)."""
    o, _ = forward(theta, F, bf16)
    lab = rotate_out(o, FR, head)
    out = np.zeros((Ns, NOUT))
    np.add.at(out, tg, lab)
    return out


def loss_and_grad(theta, F, FR, tg, labels, bf16=False, head=0):
    """Loss over the spheres that carry labels (all Ns rows of `labels`) and its
    gradient with respect to the flat parameters (plain backpropagation; with bf16
    the rounded values are used in the products and the gradient flows straight
    through the rounding)."""
    Ns = len(labels)
    P = unflatten(theta)
    rd = bf16_round if bf16 else (lambda v: v)
    o, (x0, h1, h2, h3) = forward(theta, F, bf16)
    M = head_matrices(FR, head)
    lab = np.einsum("pij,pj->pi", M, o)
    pred = np.zeros((Ns, NOUT))
    np.add.at(pred, tg, lab)
    diff = pred - labels
    loss = float((diff ** 2).sum() / (6.0 * Ns))
    dpred = 2.0 * diff / (6.0 * Ns)
    dlab = dpred[tg]
    # lab = M o  =>  do = M^T dlab
    do = np.einsum("pij,pi->pj", M, dlab)
    g = {}
    g["W4"] = do.T @ rd(h3)
    g["b4"] = do.sum(0)
    dz3 = (do @ rd(P["W4"])) * (1.0 - h3 ** 2)
    g["W3"] = dz3.T @ rd(h2)
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ rd(P["W3"])) * (1.0 - h2 ** 2)
    g["W2"] = dz2.T @ rd(h1)
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ rd(P["W2"])) * (1.0 - h1 ** 2)
    g["W1"] = dz1.T @ x0
    g["b1"] = dz1.sum(0)
    return loss, flatten(g)


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def labels_qstrain(QH_solve, QH_onebody, s0, sigma):
    """Labels [N, 6] of the strain-mode head: sigma/s0 (Q^(2s) of the solve - one-body), 0."""
    out = np.zeros((len(QH_solve), NOUT))
    out[:, :5] = sigma / s0 * (np.asarray(QH_solve, float)[:, :5] - np.asarray(QH_onebody, float)[:, :5])
    return out
