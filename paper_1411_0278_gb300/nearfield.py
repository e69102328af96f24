"""Learned near-field correction: training labels, training and evaluation.

Every step runs in libgbi's kernels; this module only orders the C-ABI calls:

* labels: for each small system the Galerkin solution at l <= 4 (gbi_batch_solve,
  Sec. II-III) and the superposition approximation at l <= 2 (gbi_batch_superpose,
  Sec. IV) of force- and torque-free spheres with V^a = vs p and
  V^(2s) = s0 (pp - I/3); gbi_mlp_labels scales their difference;
* training: gbi_mlp_train (forward, loss, backward and Adam kernels);
* use: superposition plus gbi_mlp_correct, compared with the plain solve.

A second head (gbi_mlp_set_head 1) predicts the correction of the strain-mode flow
coefficient Q^(2s) beyond its one-body value (gbi_qh_onebody); one-body Q^H plus that
correction (guess_qh) is the initial guess of a warm-started gbi_solve, so the solve --
not the network -- decides the result.

The network and its training have no counterpart in the paper.
"""
import numpy as np

from . import _native

NIN, NH, NOUT = 9, 128, 6
LAYERS = [(NH, NIN), (NH, NH), (NH, NH), (NOUT, NH)]


def init_theta(seed):
    """Glorot-uniform weights and zero biases in the flat layout of gbi_mlp_set."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in LAYERS:
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    th = np.concatenate(parts).astype(np.float32)
    assert th.size == _native.MLP_NPARAM
    return th


def _inputs(ctx, R, p, trunc, vs, s0):
    return ctx.trap_inputs(R.shape[0], trunc, 0.0, vs, s0, 0.0, R, p)


def exact_and_superposition(ctx, R, p, offsets, a, eta, vs, s0, precision=2, rtol=1e-10, chunk=20000):
    """(Vx, Ox) of the l <= 4 Galerkin solve and (Vs, Os) of the l <= 2 superposition for
    every system; the solve runs in chunks of `chunk` systems to bound the Krylov memory."""
    import torch
    N = R.shape[0]
    Vx = torch.empty((N, 3), dtype=torch.float64, device=R.device)
    Ox = torch.empty_like(Vx)
    prm4 = _native.params(a=a, eta=eta, trunc=4, precision=precision, rtol=rtol, restart=40, max_iter=4000,
                          inner_rtol=1e-5)
    nsys = len(offsets) - 1
    info = []
    for c0 in range(0, nsys, chunk):
        c1 = min(nsys, c0 + chunk)
        lo, hi = offsets[c0], offsets[c1]
        sub = [o - lo for o in offsets[c0:c1 + 1]]
        Rc, pc = R[lo:hi].contiguous(), p[lo:hi].contiguous()
        inp = _inputs(ctx, Rc, pc, 4, vs, s0)
        V, O, _, inf, _ = ctx.batch_solve(prm4, sub, Rc, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
        Vx[lo:hi] = V
        Ox[lo:hi] = O
        info.append(inf)
    prm2 = _native.params(a=a, eta=eta, trunc=2, precision=precision)
    inp = _inputs(ctx, R, p, 2, vs, s0)
    Vs, Os = ctx.batch_superpose(prm2, offsets, R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
    return Vx, Ox, Vs, Os, info


def exact_qh(ctx, R, p, offsets, a, eta, vs, s0, trunc=4, precision=2, rtol=1e-10, chunk=20000):
    """Q^H of the Galerkin solve (truncation trunc) and the one-body Q^H of every system."""
    import torch
    N = R.shape[0]
    h = _native.h(trunc)
    QHx = torch.empty((N, h), dtype=torch.float64, device=R.device)
    QH1 = torch.empty_like(QHx)
    prm = _native.params(a=a, eta=eta, trunc=trunc, precision=precision, rtol=rtol, restart=40, max_iter=4000,
                         inner_rtol=1e-5)
    nsys = len(offsets) - 1
    for c0 in range(0, nsys, chunk):
        c1 = min(nsys, c0 + chunk)
        lo, hi = offsets[c0], offsets[c1]
        sub = [o - lo for o in offsets[c0:c1 + 1]]
        Rc, pc = R[lo:hi].contiguous(), p[lo:hi].contiguous()
        inp = _inputs(ctx, Rc, pc, trunc, vs, s0)
        _, _, QH, _, _ = ctx.batch_solve(prm, sub, Rc, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
        QHx[lo:hi] = QH
        QH1[lo:hi] = ctx.qh_onebody(prm, inp["VH"])
    return QHx, QH1


def make_dataset_qh(ctx, R, p, offsets, a, eta, vs, s0, sigma=0.0, chunk=20000):
    """Training data of the strain-mode head: labels sigma/s0 (Q^(2s)_solve - one-body)."""
    QHx, QH1 = exact_qh(ctx, R, p, offsets, a, eta, vs, s0, chunk=chunk)
    labels, sigma = ctx.mlp_labels_qh(s0, QHx, QH1, sigma)
    return dict(R=R, p=p, offsets=list(offsets), a=a, eta=eta, vs=vs, s0=s0, QHx=QHx, QH1=QH1, labels=labels,
                sigma=sigma)


def train_qh(ctx, data, epochs=30, batch_systems=512, lr0=3e-3, lr1=1e-4, seed=0, theta=None):
    """The strain-mode head: select it, initialise (or take theta), train."""
    ctx.mlp_set_head(1)
    return train(ctx, data, epochs, batch_systems, lr0, lr1, seed, theta)


def guess_qh(ctx, prm, R, p, VH, s0, offsets=None, network=True):
    """Initial guess of Q^H: one-body values, plus the strain-mode head's correction."""
    QH = ctx.qh_onebody(prm, VH)
    if network:
        ctx.mlp_correct_qh(R, p, prm.a, s0, QH, offsets)
    return QH


def evaluate_qh(ctx, data):
    """Relative 2-norm error of the one-body and the learned Q^(2s) against the solve's,
    and of the whole Q^H guess."""
    QHx, QH1 = data["QHx"], data["QH1"]
    QHg = QH1.clone()
    ctx.mlp_correct_qh(data["R"], data["p"], data["a"], data["s0"], QHg, data["offsets"])

    def rel(a, b):
        return float((a - b).norm() / b.norm())
    return dict(one_body=dict(Q2s=rel(QH1[:, :5], QHx[:, :5]), QH=rel(QH1, QHx)),
                with_network=dict(Q2s=rel(QHg[:, :5], QHx[:, :5]), QH=rel(QHg, QHx)))


def make_dataset(ctx, R, p, offsets, a, eta, vs, s0, sigma=0.0, chunk=20000):
    Vx, Ox, Vs, Os, info = exact_and_superposition(ctx, R, p, offsets, a, eta, vs, s0, chunk=chunk)
    labels, sigma = ctx.mlp_labels(s0, Vx, Ox, Vs, Os, sigma)
    return dict(R=R, p=p, offsets=list(offsets), a=a, eta=eta, vs=vs, s0=s0, Vx=Vx, Ox=Ox, Vs=Vs, Os=Os,
                labels=labels, sigma=sigma, info=info)


def train(ctx, data, epochs=30, batch_systems=512, lr0=3e-3, lr1=1e-4, seed=0, theta=None):
    """Initialise (or take theta), load, and train on the dataset; returns the loss history."""
    th = init_theta(seed) if theta is None else theta
    ctx.mlp_set(th, data["sigma"])
    return ctx.mlp_train(data["R"], data["p"], data["a"], data["offsets"], data["labels"], epochs, batch_systems,
                         lr0, lr1)


def relative_errors(V, O, Vx, Ox, Va):
    """||V - Vx|| / ||Vx - Va|| and ||O - Ox|| / ||Ox|| over all spheres (2-norms)."""
    dv = float((V - Vx).norm() / (Vx - Va).norm())
    dw = float((O - Ox).norm() / Ox.norm())
    return dv, dw


def evaluate(ctx, data):
    """Errors of the superposition alone and with the network against the l <= 4 solve."""
    import torch
    Va = data["vs"] * data["p"]
    sup = relative_errors(data["Vs"], data["Os"], data["Vx"], data["Ox"], Va)
    V = data["Vs"].clone()
    O = data["Os"].clone()
    ctx.mlp_correct(data["R"], data["p"], data["a"], data["s0"], V, O, data["offsets"])
    torch.cuda.synchronize()
    net = relative_errors(V, O, data["Vx"], data["Ox"], Va)
    return dict(superposition=dict(V=sup[0], Omega=sup[1]), with_network=dict(V=net[0], Omega=net[1]))
