"""Learned near-field correction: training labels, training and evaluation.

Every step runs in libgbi's kernels; this module only orders the C-ABI calls:

* labels: for each small system the Galerkin solution at l <= 4 (gbi_batch_solve,
  Sec. II-III) and the superposition approximation at l <= 2 (gbi_batch_superpose,
  Sec. IV) of force- and torque-free spheres with V^a = vs p and
  V^(2s) = s0 (pp - I/3); gbi_mlp_labels scales their difference;
* training: gbi_mlp_train (forward, loss, backward and Adam kernels);
* use: superposition plus gbi_mlp_correct, compared with the plain solve.

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
