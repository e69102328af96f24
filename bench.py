#!/usr/bin/env python
"""Benchmark of the Galerkin boundary-integral hot path on GB300.

Workload (default): N = 1024 active spheres at volume fraction 0.05, truncation
l <= 3 (25 higher components per sphere), harmonic trap k = 0.01, V^a = 0.1 p,
V^(2s) = 0.05 (pp - I/3).  One step = trap inputs from (R, p), the full
traction solve (right-hand-side pass, restarted GMRES with FP32 pair sums and
FP64 Arnoldi, iterative refinement to ||b - A q|| / ||b|| <= 1e-10, output pass)
and one forward-Euler update, all inside libgbi.

Metric: pair-interactions/s (ordered pairs summed over every pair pass of the
step) and solves/s.  Also reported: the roofline of the dominant kernel, the
end-to-end number through the host-pointer C-ABI call, every precision mode of
the same solve with its residual against the FP64 system, the N = 64 FP64
trajectory (100 re-solved Euler steps), the N = 10^4 superposition trajectory
(10^4 steps and its steady convective flux), the batched and learned workloads,
and the FP64 CPU oracle timed on bounded samples on this machine's cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank solves its own replica of the workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pair-interactions/s & Galerkin solves/s at stated error vs FP64; % FP32 peak"
UNIT = "pair-interactions/s"
FP64_NOMINAL_TFLOPS = 1.25          # GB300 FP64 (recipe's nominal figure)
FP32_LANES = 128                    # FP32 lanes per SM (Blackwell)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_alu_peak_tflops(sm_mhz, sms):
    """FP32 CUDA-core peak: SMs x 128 lanes x 2 flops (FMA) x clock."""
    return sms * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle baseline

def oracle_pair_rate(R, trunc, a, npairs, seed=0):
    """FP64 oracle (dense pair blocks + apply) on a sample of ordered pairs: pairs/s."""
    import numpy as np

    from oracle import galerkin
    rng = np.random.default_rng(seed)
    N = len(R)
    n = rng.integers(0, N, size=npairs)
    m = (n + rng.integers(1, N, size=npairs)) % N
    d = galerkin.ModeBasis(trunc).d
    x = rng.normal(size=(npairs, d))
    galerkin.pair_blocks(R[:2] - R[1:3], a, trunc)        # warm the weight tables
    t0 = time.perf_counter()
    blocks = galerkin.pair_blocks(R[n] - R[m], a, trunc)
    y = np.einsum("kpq,kq->kp", blocks, x)
    dt = time.perf_counter() - t0
    assert np.all(np.isfinite(y))
    return npairs / dt, dt


def oracle_baselines(c1, c2, c3, npairs=12000):
    """The FP64 oracle, as it stands, on bounded samples of three workloads, on this host's
    cores: dense pair blocks (the unit of the headline metric), a whole N = 64 dense solve,
    the N = 1024 dense solve extrapolated from its parts, and the N = 10^4 superposition sum
    for sampled spheres."""
    import numpy as np

    from oracle import dynamics, galerkin
    rate3, dt3 = oracle_pair_rate(c2["R"], c2["trunc"], c2["a"], npairs)
    trap = lambda c: dict(a=c["a"], eta=c["eta"], k=c["k"], vs=c["vs"], s0=c["s0"], d0=c["d0"])
    # N = 64, l <= 2: assemble the dense system, LU, outputs
    dynamics.velocities(c1["R"][:4], c1["p"][:4], trap(c1), c1["trunc"], False)
    t0 = time.perf_counter()
    dynamics.velocities(c1["R"], c1["p"], trap(c1), c1["trunc"], False)
    t1 = time.perf_counter() - t0
    # N = 1024, l <= 3: N(N-1) dense pair blocks at the sampled rate, plus the LU of the
    # n = N h system scaled as n^3 from a timed LU of a smaller dense system
    N2 = len(c2["R"])
    n2 = N2 * 25
    ns = 2400
    rng = np.random.default_rng(0)
    M = rng.normal(size=(ns, ns))
    M = M @ M.T + ns * np.eye(ns)
    rhs = rng.normal(size=ns)
    t0 = time.perf_counter()
    np.linalg.solve(M, rhs)
    t_lu_s = time.perf_counter() - t0
    t_asm2 = N2 * (N2 - 1) / rate3
    t_lu2 = t_lu_s * (n2 / ns) ** 3
    # N = 10^4, l <= 2 superposition: the oracle's pair sum for sampled target spheres
    N3 = len(c3["R"])
    tg = np.arange(0, N3, N3 // 6)[:6]
    inp3 = dynamics.trap_inputs(c3["R"], c3["p"], trap(c3), 2)
    t0 = time.perf_counter()
    galerkin.superpose(c3["R"], inp3["Va"], inp3["Oa"], inp3["VH"], inp3["Fe"], inp3["Te"], c3["a"], c3["eta"], 2,
                       targets=tg)
    t3 = time.perf_counter() - t0
    rate_sup = len(tg) * (N3 - 1) / t3
    return {"value": rate3, "unit": UNIT, "cores": blas_threads(), "kind": "oracle", "cpu_model": cpu_model(),
            "sample": "%d random ordered pairs of the N=1024 l<=3 suspension, dense FP64 31x31 pair blocks + "
                      "apply (%.1f s)" % (npairs, dt3),
            "solve_N64_l2": {"solves_per_s": 1.0 / t1, "s_per_solve": t1, "how": "whole dense assembly + LU + "
                             "outputs of the N=64 l<=2 suspension (n = 512 unknowns), timed"},
            "solve_N1024_l3": {"solves_per_s": 1.0 / (t_asm2 + t_lu2), "s_per_solve": t_asm2 + t_lu2,
                               "assembly_s": t_asm2, "lu_s": t_lu2,
                               "how": "extrapolated: N(N-1) pair blocks at the sampled rate, plus LU of n = %d "
                                      "scaled as n^3 from a timed LU of n = %d (%.2f s)" % (n2, ns, t_lu_s)},
            "superposition_N10000": {"pairs_per_s": rate_sup, "s_per_step": N3 * (N3 - 1) / rate_sup,
                                     "how": "oracle superposition sum for %d sampled spheres against all N-1 "
                                            "sources (%.1f s), extrapolated to one step of all N" % (len(tg), t3)}}


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        n = [i.get("num_threads") for i in info if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count()


# ----------------------------------------------------------------------------- distributed

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import workloads
    c = workloads.config2()
    npairs = 1500
    for _ in range(args.warmup):
        oracle_pair_rate(c["R"], 3, c["a"], 200)
    total_pairs, total_t = 0, 0.0
    for k in range(args.steps):
        rate, dt = oracle_pair_rate(c["R"], 3, c["a"], npairs, seed=k)
        total_pairs += npairs
        total_t += dt
    value = total_pairs / total_t
    cores = blas_threads()
    sample = "%d random ordered pairs of the N=1024 l<=3 suspension per step (dense 31x31 pair blocks + apply)" % npairs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": c["name"], "N": 1024, "trunc": 3},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# passes timed by gbi_tune, in the order of its result
TUNED_PASSES = ["HH_f32", "HH_df", "HL_df", "Lall_df", "HL_f32", "Lall_f32"]
RESET_EVERY = 20     # timed trap steps between returns to the initial suspension
CLASS_PASS = {"H": 2, "L": 1, "all": 0}


def learned_nearfield(ctx, gbi, dev, stream, peaks):
    """Learned near-field correction: label generation and training on 2- and 3-sphere
    systems, errors against the plain l <= 4 solve (held-out systems and a dense
    2000-sphere suspension), and the N = 10^5 evaluation (superposition + network)."""
    import time
    import torch
    import workloads
    from paper_1411_0278_gb300 import nearfield

    def T(x):
        return torch.tensor(x, dtype=torch.float64, device=dev)

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=1):
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for _ in range(reps):
            out = fn()
        ev1.record(stream)
        ev1.synchronize()
        return out, ev0.elapsed_time(ev1) / reps

    tr = workloads.nearfield_systems(100000, 100000, k=20)
    a, eta, vs, s0 = 1.0, tr["eta"], tr["vs"], tr["s0"]
    t0 = time.time()
    dtr = nearfield.make_dataset(ctx, T(tr["R"]), T(tr["p"]), tr["offsets"], a, eta, vs, s0)
    torch.cuda.synchronize(dev)
    t_label = time.time() - t0
    epochs = 40
    t0 = time.time()
    hist = nearfield.train(ctx, dtr, epochs=epochs, batch_systems=1024, lr0=3e-3, lr1=3e-5, seed=1)
    t_train = time.time() - t0
    held = {}
    for name, n2, n3 in (("two_body", 1000, 0), ("three_body", 0, 1000)):
        te = workloads.nearfield_systems(n2, n3, k=21)
        dte = nearfield.make_dataset(ctx, T(te["R"]), T(te["p"]), te["offsets"], a, eta, vs, s0,
                                     sigma=dtr["sigma"])
        held[name] = nearfield.evaluate(ctx, dte)

    # dense suspension: plain l <= 4 solve against superposition (+ network)
    ss = workloads.suspension(2000, 0.1, 2.05, workloads.SEED_BASE + 5200)
    Rs, ps = T(ss["R"]), T(ss["p"])
    i4 = ctx.trap_inputs(2000, 4, 0.0, vs, s0, 0.0, Rs, ps)
    i2 = ctx.trap_inputs(2000, 2, 0.0, vs, s0, 0.0, Rs, ps)
    prm4 = gbi.params(a=a, eta=eta, trunc=4, precision=2, rtol=1e-10, restart=40, max_iter=2000, inner_rtol=1e-5)
    prm2 = gbi.params(a=a, eta=eta, trunc=2, precision=1)
    ctx.tune(4, [0, 2000])
    (Vx, Ox, _, ix, _), ms_exact = timed(lambda: ctx.solve(prm4, Rs, i4["Va"], i4["Oa"], i4["VH"], i4["Fe"], i4["Te"]))

    def learned():
        V, O = ctx.superpose(prm2, Rs, i2["Va"], i2["Oa"], i2["VH"], i2["Fe"], i2["Te"])
        ctx.mlp_correct(Rs, ps, a, s0, V, O)
        return V, O
    learned()
    (Vl, Ol), ms_learned = timed(learned, 3)
    Vsup, Osup = ctx.superpose(prm2, Rs, i2["Va"], i2["Oa"], i2["VH"], i2["Fe"], i2["Te"])
    torch.cuda.synchronize(dev)
    Va = i2["Va"]
    dense = {"N": 2000, "superposition": dict(zip(("V", "Omega"), nearfield.relative_errors(Vsup, Osup, Vx, Ox, Va))),
             "with_network": dict(zip(("V", "Omega"), nearfield.relative_errors(Vl, Ol, Vx, Ox, Va))),
             "exact_ms": ms_exact, "exact_iters": ix.iters, "exact_rel_residual": ix.rel_residual,
             "learned_ms": ms_learned, "speedup_learned_vs_exact": ms_exact / ms_learned}

    # N = 10^5: superposition (closed-form l <= 2 kernel, FP32) plus the network
    c5 = workloads.config5()
    N5 = len(c5["R"])
    R5, p5 = T(c5["R"]), T(c5["p"])
    in5 = ctx.trap_inputs(N5, 2, 0.0, vs, s0, 0.0, R5, p5)
    V5 = torch.empty((N5, 3), dtype=torch.float64, device=dev)
    O5 = torch.empty_like(V5)
    npairs = [0]

    def full():
        ctx.superpose(prm2, R5, in5["Va"], in5["Oa"], in5["VH"], in5["Fe"], in5["Te"], V5, O5)
        npairs[0] = ctx.mlp_correct(R5, p5, a, s0, V5, O5)
    full()
    _, ms_full = timed(full, 3)
    # the network alone on the same pairs
    tg, sr = ctx.pairs(R5, a, 4.0)
    F, FR = ctx.mlp_features(R5, p5, tg, sr, a)
    engines = {}
    for eng in (0, 1):
        ctx.mlp_set_engine(eng)
        ctx.mlp_forward(F, FR)
        _, engines[eng] = timed(lambda: ctx.mlp_forward(F, FR), 10)
        ctx.mlp_status()
    ctx.mlp_set_engine(1)
    ms_net = engines[1]
    P = int(tg.shape[0])
    flops_net = 2.0 * (9 * 128 + 2 * 128 * 128 + 128 * 6) * P
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    pairs5 = N5 * (N5 - 1) + P
    warm = learned_warm_start(ctx, gbi, T, timed, a, eta, vs, s0, c5)
    return {"workload": c5["name"], "N": N5, "value": pairs5 / (ms_full / 1e3), "unit": UNIT,
            "ms_per_evaluation": ms_full, "network_pairs": P, "warm_start_at_equal_error": warm,
            "network": {"ms": ms_net, "achieved_tflops": flops_net / (ms_net / 1e3) / 1e12,
                        "peak_bf16_tflops": bf16_peak,
                        "frac": flops_net / (ms_net / 1e3) / 1e12 / bf16_peak,
                        "kernel": "k_infer_tc (tcgen05.mma kind::f16, M128 N128 K16, accumulator in tensor "
                                  "memory)",
                        "ms_mma_sync_kernel": engines[0]},
            "training": {"systems": len(tr["offsets"]) - 1, "spheres": len(tr["R"]), "label_s": t_label,
                         "train_s": t_train, "epochs": epochs, "loss_first": hist[0], "loss_last": hist[-1],
                         "sigma": dtr["sigma"]},
            "heldout": held, "dense_suspension": dense,
            "note": "errors are relative to the plain l<=4 Galerkin solve: ||V - Vx|| / ||Vx - Va||, "
                    "||Omega - Ox|| / ||Ox||"}



def learned_warm_start(ctx, gbi, T, timed, a, eta, vs, s0, c5):
    """The strain-mode head as a warm start of the l <= 4 solve, at equal velocity error.

    Trains head 1 on 2- and 3-sphere systems (labels: Q^(2s) of the l <= 4 solve minus the
    one-body value), then solves dense suspensions -- the 2000-sphere one (volume fraction
    0.1, 2.05a exclusion) and the 5000 spheres of the N = 10^5 workload nearest its centre --
    in several forms: plain FP64 GMRES from zero, mixed precision from zero, from the
    one-body Q^H and from the learned guess (the guess's own time included).  Each form
    runs at each of a few (refinement tolerance, inner tolerance) settings and reports
    the fastest one whose velocity error is at most 1e-6: max_n |V_n - V_n,ref| /
    max_n |V_n,ref - V^a_n| against an FP64 solve to 1e-12."""
    import time
    import numpy as np
    import torch
    import workloads
    from paper_1411_0278_gb300 import nearfield

    tr = workloads.nearfield_systems(40000, 40000, k=30)
    t0 = time.time()
    dtr = nearfield.make_dataset_qh(ctx, T(tr["R"]), T(tr["p"]), tr["offsets"], a, eta, vs, s0)
    torch.cuda.synchronize()
    t_label = time.time() - t0
    t0 = time.time()
    hist = nearfield.train_qh(ctx, dtr, epochs=40, batch_systems=512, lr0=3e-3, lr1=3e-5, seed=3)
    t_train = time.time() - t0
    te = workloads.nearfield_systems(1000, 1000, k=31)
    held = nearfield.evaluate_qh(ctx, nearfield.make_dataset_qh(ctx, T(te["R"]), T(te["p"]), te["offsets"], a, eta,
                                                                vs, s0, sigma=dtr["sigma"]))
    ss = workloads.suspension(2000, 0.1, 2.05, workloads.SEED_BASE + 5200)
    R5 = np.asarray(c5["R"])
    near = np.argsort(np.linalg.norm(R5 - R5.mean(axis=0), axis=1))[:5000]
    cases = [("N2000_phi0.1", ss["R"], ss["p"]), ("config5_central_5000", R5[near], np.asarray(c5["p"])[near])]
    settings = {0: [(1e-6, 0.0), (1e-7, 0.0)], 2: [(1e-6, 1e-5), (1e-6, 1e-6), (1e-7, 1e-5)],
                3: [(1e-6, 1e-5), (1e-6, 1e-6), (1e-7, 1e-5)]}
    out = {"target_V_error": 1e-6,
           "training": {"systems": len(tr["offsets"]) - 1, "label_s": t_label, "train_s": t_train,
                        "loss_first": hist[0], "loss_last": hist[-1], "sigma": dtr["sigma"]},
           "heldout_Q2s_error": held, "cases": {}}
    for name, Rn, pn in cases:
        N = len(Rn)
        R, p = T(Rn), T(pn)
        inp = ctx.trap_inputs(N, 4, 0.0, vs, s0, 0.0, R, p)
        args = (R, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
        ref = gbi.params(a=a, eta=eta, trunc=4, precision=0, rtol=1e-12, restart=40, max_iter=4000)
        Vr = ctx.solve(ref, *args)[0]
        scale = float((Vr - inp["Va"]).norm(dim=1).max())
        forms = {}
        for form, prec, guess in (("fp64_gmres_from_zero", 0, None), ("mixed2_from_zero", 2, None),
                                  ("mixed2_from_one_body", 2, "one_body"), ("mixed2_from_learned", 2, "learned"),
                                  ("mixed3_from_zero", 3, None), ("mixed3_from_learned", 3, "learned")):
            tried = []
            for rtol, inner in settings[prec]:
                prm = gbi.params(a=a, eta=eta, trunc=4, precision=prec, rtol=rtol, restart=40, max_iter=4000,
                                 inner_rtol=inner if inner > 0 else 1e-5)

                def run():
                    if guess is None:
                        return ctx.solve(prm, *args)
                    Q0 = nearfield.guess_qh(ctx, prm, R, p, inp["VH"], s0, network=(guess == "learned"))
                    return ctx.solve(prm, *args, QH=Q0, warm_start=True)
                reps = 1 if prec == 0 else 3
                if prec != 0:
                    run()                       # first call: the host-driven sequence
                run()                           # a repeat: builds (then replays) the solve graph
                (V, _, _, info, _), ms = timed(run, reps)
                err = float((V - Vr).norm(dim=1).max()) / scale
                tried.append({"rtol": rtol, "inner_rtol": inner if prec else None, "ms": ms, "V_error": err,
                              "iters": info.iters, "refinements": info.refinements,
                              "rel_residual": info.rel_residual})
            ok = [t for t in tried if t["V_error"] <= 1e-6]
            best = min(ok, key=lambda t: t["ms"]) if ok else None
            forms[form] = {"best": best, "solves_per_s": 1e3 / best["ms"] if best else None, "settings": tried}
        base = forms["fp64_gmres_from_zero"]["best"]["ms"]
        for f in forms.values():
            f["speedup_vs_fp64_gmres"] = base / f["best"]["ms"] if f["best"] else None
        out["cases"][name] = {"N": N, "forms": forms,
                              "learned_vs_mixed_from_zero": {
                                  "precision2": forms["mixed2_from_zero"]["best"]["ms"] /
                                  forms["mixed2_from_learned"]["best"]["ms"],
                                  "precision3": forms["mixed3_from_zero"]["best"]["ms"] /
                                  forms["mixed3_from_learned"]["best"]["ms"]}}
    return out


def h_mode_slices(trunc):
    """(name, first column, width) of every higher mode l-sigma in the packed [N][h] layout of
    V^H and Q^H: the modes after 1s and 2a, each 2(l - sigma) + 1 wide."""
    from paper_1411_0278_gb300 import gen_tables
    out, off = [], 0
    for name, L, sig in gen_tables.MODES[2:gen_tables.NMODES[trunc]]:
        k = 2 * (L - sig) + 1
        out.append((name, off, k))
        off += k
    return out


def job_totals(t_local, pairs_local, world, device):
    """Whole-job time (the slowest rank) and work (summed over ranks) of a timed region."""
    if world <= 1:
        return t_local, float(pairs_local)
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    w = torch.tensor([float(pairs_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t[0]), float(w[0])


def fp64_system_residual(ctx, gbi, N, trunc, a, eta, R, inp, QH):
    """||b - A q|| / ||b|| of the FP64 system for a solution Q^H: b = -8 pi eta V^H - G^HL F^L
    and A = G^HH (pair and self terms), both evaluated by the FP64 pair kernel, in the
    solver's internal coordinates (x = c y per component)."""
    import torch
    sc = torch.tensor(gbi.component_scales(trunc), dtype=torch.float64, device=R.device)
    h = len(sc) - 6
    xV = (inp["VH"] * sc[6:]).T.contiguous()
    xQ = (QH * sc[6:]).T.contiguous()
    F, T, c2a = inp["Fe"], inp["Te"], float(sc[3])
    xF = torch.stack([-F[:, 1], -F[:, 2], -F[:, 0], -c2a * T[:, 1] / a, -c2a * T[:, 2] / a,
                      -c2a * T[:, 0] / a]).contiguous()
    y1 = torch.zeros((h, N), dtype=torch.float64, device=R.device)
    y2 = torch.zeros_like(y1)
    ctx.apply(N, trunc, a, gbi.SET_H, gbi.SET_L, 0, R, xF, y1, 1.0, 0.0, False)
    ctx.apply(N, trunc, a, gbi.SET_H, gbi.SET_H, 0, R, xQ, y2, 1.0, 0.0, True)
    b = -8.0 * math.pi * eta * xV - y1
    return float((b - y2).norm() / b.norm())


def pass_launch_time(ctx, gbi, N, trunc, a, R, cls, reps=40):
    """Average duration of one launch of pair-pass class cls (precision * 9 + rows * 3 + cols)
    with the tuned form: reps back-to-back launches through gbi_apply, CUDA events around each
    pair kernel on the library stream (the host runs ahead, so no launch gap is timed)."""
    import torch
    prec, rows, cols = cls // 9, (cls % 9) // 3, cls % 3
    D = gbi.d(trunc)
    nr = {0: D, 1: 6, 2: D - 6}[rows]
    nc = {0: D, 1: 6, 2: D - 6}[cols]
    x = torch.randn((nc, N), dtype=torch.float64, device=R.device)
    y = torch.zeros((nr, N), dtype=torch.float64, device=R.device)
    self_ok = rows == cols or (rows == 1 and cols == 0)
    for _ in range(3):
        ctx.apply(N, trunc, a, rows, cols, prec, R, x, y, 1.0, 0.0, self_ok)
    ctx.set_profiling(True)
    for _ in range(reps):
        ctx.apply(N, trunc, a, rows, cols, prec, R, x, y, 1.0, 0.0, self_ok)
    st = ctx.kernel_stats(cls)
    ctx.set_profiling(False)
    return st["ms"] / max(1, st["launches"]), st["flops"] / max(1, st["launches"])


def precision_lines(ctx, gbi, c, R0, inp, flush, stream):
    """The headline solve (N = 1024, l <= 3, cold start, rtol 1e-10) in every precision mode:
    ms per solve and solves/s (CUDA events, L2 flushed before each solve), the residual
    against the FP64 system, and V, Omega, Q^H (per mode) against the all-FP64 solve."""
    import torch
    N, trunc = len(c["R"]), c["trunc"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    args = (inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
    sols, out = {}, {}
    names = {0: "FP64 throughout", 1: "FP32 pair sums in GMRES; FP64 right-hand side, refinement residuals, "
             "outputs", 2: "FP32 pair sums in GMRES; double-float right-hand side, refinement residuals, outputs",
             3: "FP32 pair sums in GMRES, right-hand side and outputs; double-float refinement residuals"}
    for pr in (0, 1, 2, 3):
        prm = gbi.params(a=c["a"], eta=c["eta"], trunc=trunc, precision=pr, rtol=1e-10, restart=40, inner_rtol=1e-5,
                         min_sep=2.0)
        for _ in range(2):
            ctx.solve(prm, R0, *args)
        reps = 3 if pr == 0 else 10
        tot = 0.0
        for _ in range(reps):
            flush.fill_(1.0)
            ev0.record(stream)
            V, O, Q, info, _ = ctx.solve(prm, R0, *args)
            ev1.record(stream)
            ev1.synchronize()
            tot += ev0.elapsed_time(ev1)
        sols[pr] = (V.clone(), O.clone(), Q.clone(), info)
        out["p%d" % pr] = {"precision": names[pr], "ms_per_solve": tot / reps, "solves_per_s": 1e3 * reps / tot,
                           "iters": info.iters, "refinements": info.refinements,
                           "solver_rel_residual": info.rel_residual,
                           "residual_vs_fp64_system": fp64_system_residual(ctx, gbi, N, trunc, c["a"], c["eta"], R0,
                                                                           inp, Q)}

    def rel(x, y):
        return float((x - y).abs().max() / y.abs().max())
    V0, O0, Q0, _ = sols[0]
    for pr in (1, 2, 3):
        V, O, Q, _ = sols[pr]
        out["p%d" % pr].update({"V_rel_vs_fp64": rel(V, V0), "Omega_rel_vs_fp64": rel(O, O0),
                                "QH_rel_vs_fp64": rel(Q, Q0),
                                "QH_rel_per_mode": {nm: rel(Q[:, o:o + k], Q0[:, o:o + k])
                                                    for nm, o, k in h_mode_slices(trunc)},
                                "speedup_vs_fp64": out["p0"]["ms_per_solve"] / out["p%d" % pr]["ms_per_solve"]})
    out["note"] = ("residual_vs_fp64_system = ||b - A q|| / ||b|| with b and A of the FP64 system (FP64 pair "
                   "kernel); solver_rel_residual is the solver's own refinement residual, whose right-hand side "
                   "is FP32-summed in precision 3")
    return out


def trajectory_n64(ctx, gbi, dev, stream):
    """N = 64, l <= 2: one FP64 solve to 1e-10, then 100 forward-Euler steps of dt = 0.1, each
    re-solved in FP64 (warm-started from the previous step's Q^H), through gbi_trap_step."""
    import torch
    import workloads
    c = workloads.config1()
    N = len(c["R"])
    prm = gbi.params(a=c["a"], eta=c["eta"], trunc=c["trunc"], precision=0, rtol=c["rtol"], restart=40)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    R0 = torch.tensor(c["R"], dtype=torch.float64, device=dev)
    p0 = torch.tensor(c["p"], dtype=torch.float64, device=dev)
    inp = ctx.trap_inputs(N, c["trunc"], c["k"], c["vs"], c["s0"], c["d0"], R0, p0)
    for _ in range(2):
        ctx.solve(prm, R0, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
    ev0.record(stream)
    _, _, _, i0, _ = ctx.solve(prm, R0, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
    ev1.record(stream)
    ev1.synchronize()
    ms_solve = ev0.elapsed_time(ev1)
    R, p = R0.clone(), p0.clone()
    ev0.record(stream)
    info = ctx.trap_step(prm, R, p, c["dt"], c["k"], c["vs"], c["s0"], c["d0"], False, c["steps"])
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    d = torch.cdist(R, R) + torch.eye(N, dtype=torch.float64, device=dev) * 1e9
    return {"workload": c["name"], "N": N, "trunc": c["trunc"], "precision": "FP64 throughout", "dt": c["dt"],
            "first_solve_ms": ms_solve, "first_solve_iters": i0.iters, "first_solve_rel_residual": i0.rel_residual,
            "steps": c["steps"], "ms_total": ms, "steps_per_s": 1e3 * c["steps"] / ms,
            "solves_per_s": 1e3 * c["steps"] / ms, "gmres_iters_per_step": info.iters / c["steps"],
            "max_rel_residual": info.rel_residual, "pair_interactions_per_s": info.pair_interactions / (ms / 1e3),
            "min_separation_a_final": float(d.min()) / c["a"],
            "start": "each step warm-started from the previous step's Q^H"}


def trajectory_trap(ctx, gbi, dev, stream, R_init, p_init, k_trap, steps, dt, tail=0.2, every=10, vs=0.1, s0=0.05):
    """Superposition trap dynamics (closed-form l <= 2 pair sum in FP32, forward Euler): the
    first (1 - tail) of the steps in one gbi_trap_step call (timed), then the tail in short
    calls that sample the convective flux: <v . e> over the spheres inside R*/2, e the unit
    mean orientation of those spheres, v = (R_{k+1} - R_k) / dt (exact for forward Euler),
    averaged over the samples."""
    import torch
    import workloads
    a, eta = 1.0, workloads.ETA_DEFAULT
    N = len(R_init)
    Rstar = 6 * math.pi * eta * vs * a / k_trap
    prm = gbi.params(a=a, eta=eta, trunc=2, precision=1)
    R = torch.tensor(R_init, dtype=torch.float64, device=dev)
    p = torch.tensor(p_init, dtype=torch.float64, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx.trap_step(prm, R.clone(), p.clone(), dt, k_trap, vs, s0, 0.0, True, 3)     # warm-up on a copy
    n_main = int(round(steps * (1 - tail)))
    ev0.record(stream)
    ctx.trap_step(prm, R, p, dt, k_trap, vs, s0, 0.0, True, n_main)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    flux, inner = [], []
    done = n_main
    while done < steps:
        Rk = R.clone()
        pk = p.clone()
        ctx.trap_step(prm, R, p, dt, k_trap, vs, s0, 0.0, True, 1)
        v = (R - Rk) / dt
        sel = Rk.norm(dim=1) < Rstar / 2
        if int(sel.sum()) > 0:
            e = pk[sel].mean(dim=0)
            if float(e.norm()) > 0:
                e = e / e.norm()
                flux.append(float((v[sel] @ e).mean()))
                inner.append(int(sel.sum()))
        n = min(every - 1, steps - done - 1)
        if n > 0:
            ctx.trap_step(prm, R, p, dt, k_trap, vs, s0, 0.0, True, n)
        done += 1 + max(n, 0)
    torch.cuda.synchronize(dev)
    r = R.norm(dim=1)
    return {"N": N, "dt": dt, "k_trap": k_trap, "R_star_a": Rstar / a, "steps": steps,
            "timed_steps": n_main, "ms_timed": ms, "steps_per_s": 1e3 * n_main / ms,
            "value": n_main * N * (N - 1) / (ms / 1e3), "unit": UNIT,
            "steady_convective_flux": (sum(flux) / len(flux)) if flux else None,
            "flux_samples": len(flux), "mean_inner_spheres": (sum(inner) / len(inner)) if inner else 0,
            "radius_median_a": float(r.median()) / a, "radius_max_a": float(r.max()) / a,
            "escaped_fraction": float((r > 10 * Rstar).double().mean()),
            "overlaps_note": "the superposition model has no contact force (as in the paper's trap model): "
                             "spheres may overlap, where the far-field pair formulas give large velocities",
            "flux_definition": "<v . e> over spheres with |R| < R*/2, e = unit mean orientation of those spheres, "
                               "sampled every %d steps over the last %d%% of steps" % (every, int(100 * tail))}


def squirmer_pair_orbits(ctx, gbi, dev, stream):
    """Two squirmers in a harmonic trap (Sec. V, two-particle discussion): both on the sphere
    R* = 12.56 a, pointing outwards, the second at theta0 from the first; superposition
    dynamics (l <= 2, FP32) for 40 rotational times tau_r = 8 pi eta a / k.  Reported per
    theta0: the range of the angle between the particles, their largest change of
    orientation (zero for the frozen theta0 = 180 degrees) and how often the angle turns."""
    import torch
    import workloads
    B1, B2, Rs = 0.15, -1.0 / 12.0, 12.56
    eta = workloads.ETA_DEFAULT
    k = 6 * math.pi * eta * (2 * B1 / 3) / Rs
    tau_r = 8 * math.pi * eta / k
    dt = 0.5
    every = 50
    nsteps = int(40 * tau_r / dt) // every * every
    prm = gbi.params(a=1.0, eta=eta, trunc=2, precision=1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"B1": B1, "B2": B2, "R_star_a": Rs, "k_trap": k, "tau_r": tau_r, "dt": dt, "steps": nsteps}
    total_ms = 0.0
    for th in (180.0, 115.0, 190.0, 260.0):
        t = math.radians(th)
        u = [[0.0, 0.0, 1.0], [math.sin(t), 0.0, math.cos(t)]]
        R = torch.tensor(u, dtype=torch.float64, device=dev) * Rs
        p = torch.tensor(u, dtype=torch.float64, device=dev)
        p0 = p.clone()
        angles, rot = [], 0.0
        for _ in range(nsteps // every):
            ev0.record(stream)
            ctx.squirmer_step(prm, R, p, dt, k, B1, B2, True, every)
            ev1.record(stream)
            ev1.synchronize()
            total_ms += ev0.elapsed_time(ev1)
            c = float((R[0] @ R[1]) / (R[0].norm() * R[1].norm()))
            angles.append(math.degrees(math.acos(max(-1.0, min(1.0, c)))))
            rot = max(rot, float((p - p0).abs().max()))
        d = [b - a for a, b in zip(angles, angles[1:])]
        turns = sum(1 for a, b in zip(d, d[1:]) if a * b < 0)
        out["theta0_%d" % int(th)] = {"angle_min_deg": min(angles), "angle_max_deg": max(angles),
                                      "angle_final_deg": angles[-1], "max_orientation_change": rot,
                                      "angle_turning_points": turns,
                                      "radius_final_a": [float(R[0].norm()), float(R[1].norm())]}
    out["steps_per_s"] = 4 * nsteps / (total_ms / 1e3)
    return out


def run_ours(args):
    import numpy as np
    import torch

    import paper_1411_0278_gb300 as gbi
    import workloads

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # a non-default stream lets the library replay its solves from CUDA graphs
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = gbi.Context(local, stream=stream)

    c = workloads.config2()
    N, trunc = len(c["R"]), c["trunc"]
    dt = 0.1
    # min_sep: the overlap guard (centres closer than 2a fail the step instead of being timed)
    prm = gbi.params(a=c["a"], eta=c["eta"], trunc=trunc, precision=args.precision, rtol=1e-10, restart=40,
                     inner_rtol=1e-5, min_sep=2.0)
    R0 = torch.tensor(c["R"], dtype=torch.float64, device=dev)
    p0 = torch.tensor(c["p"], dtype=torch.float64, device=dev)
    R, p = R0.clone(), p0.clone()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def step():
        return ctx.trap_step(prm, R, p, dt, c["k"], c["vs"], c["s0"], c["d0"], False, 1)

    # ---- pair-kernel tuning (form and warps per target of each pass), outside the timed region
    tuned = ctx.tune(trunc, [0, N])

    # ---- accuracy and speed of every precision mode (outside the timed region)
    inp = ctx.trap_inputs(N, trunc, c["k"], c["vs"], c["s0"], c["d0"], R0, p0)
    modes = precision_lines(ctx, gbi, c, R0, inp, flush, stream)
    head = modes["p%d" % args.precision]
    err = {"V_rel": head.get("V_rel_vs_fp64", 0.0), "Omega_rel": head.get("Omega_rel_vs_fp64", 0.0),
           "QH_rel": head.get("QH_rel_vs_fp64", 0.0), "QH_rel_per_mode": head.get("QH_rel_per_mode", {}),
           "solver_rel_residual": head["solver_rel_residual"],
           "residual_vs_fp64_system": head["residual_vs_fp64_system"]}
    vs_fp64 = {"fp64_solves_per_s": modes["p0"]["solves_per_s"], "mixed_solves_per_s": head["solves_per_s"],
               "fp64_ms_per_solve": modes["p0"]["ms_per_solve"], "mixed_ms_per_solve": head["ms_per_solve"],
               "speedup": modes["p0"]["ms_per_solve"] / head["ms_per_solve"],
               "mixed_V_rel_vs_fp64": err["V_rel"], "rtol": 1e-10,
               "note": "same input (the initial N=1024 suspension), cold start, solve only (no trap step)"}

    # ---- warm-up
    for _ in range(max(3, args.warmup)):
        step()
    R.copy_(R0)
    p.copy_(p0)
    barrier()

    # ---- timed region (no per-kernel instrumentation: graphs replayed)
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = ctx.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    step_stats = {"iters": 0, "refinements": 0, "matvecs_f32": 0, "matvecs_hp": 0, "max_residual": 0.0}

    def run_steps(k, stats=None):
        ms, pr = 0.0, 0
        for i in range(k):
            if i > 0 and i % RESET_EVERY == 0:
                # back to the initial suspension (outside the timed interval): every step
                # then starts within RESET_EVERY steps of it, whatever the step count
                R.copy_(R0)
                p.copy_(p0)
            flush.fill_(1.0)                    # evict the L2 between timed steps
            ev0.record(stream)
            info = step()
            ev1.record(stream)
            ev1.synchronize()
            ms += ev0.elapsed_time(ev1)
            pr += info.pair_interactions
            if stats is not None:
                stats["iters"] += info.iters
                stats["refinements"] += info.refinements
                stats["matvecs_f32"] += info.matvecs_f32
                stats["matvecs_hp"] += info.matvecs_f64
                stats["max_residual"] = max(stats["max_residual"], info.rel_residual)
        return ms, pr

    barrier()
    total_ms, pairs = run_steps(args.steps, step_stats)
    barrier()
    launches = ctx.kernel_launches() - launches0
    clocks = sampler.stop()
    # ---- the same steps again with CUDA events around every pair pass (direct launches):
    # which pass class dominates the step, and its share
    R.copy_(R0)
    p.copy_(p0)
    for _ in range(2):
        step()
    ctx.set_profiling(True)
    prof_ms, _ = run_steps(args.steps)
    stats = {cls: ctx.kernel_stats(cls) for cls in range(gbi._native.N_KERNEL_CLASSES)}
    ctx.set_profiling(False)

    t_job, pairs_job = job_totals(total_ms / 1e3, pairs, world, dev)
    value = pairs_job / t_job
    solves_per_s = world * args.steps / t_job

    # ---- dominant kernel and its roofline: its launch timed back to back with the tuned form
    peaks, peak_src = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = fp32_alu_peak_tflops(sm_max, sms)
    tname = {0: "double", 1: "float", 2: "double-float"}
    sname = {0: "all", 1: "L", 2: "H"}
    names = {pr * 9 + r * 3 + cc: "pair pass <l%d, rows %s, cols %s, %s>" % (trunc, sname[r], sname[cc], tname[pr])
             for pr in range(3) for r in range(3) for cc in range(3)}
    names[27] = "trap pass FP64"
    names[28] = "trap pass FP32"
    total_pass_ms = sum(v["ms"] for v in stats.values())
    dom = max(stats, key=lambda k: stats[k]["ms"])
    in_step_ms = stats[dom]["ms"] / max(1, stats[dom]["launches"])
    avg_ms, flops_per_launch = pass_launch_time(ctx, gbi, N, trunc, c["a"], R0, dom)
    achieved = flops_per_launch / (avg_ms * 1e-3) / 1e12
    is_f32 = dom == 28 or (9 <= dom < 27)       # FP32 and double-float classes run on the FP32 pipe
    peak = fp32_peak if is_f32 else FP64_NOMINAL_TFLOPS
    prec_d, rows_d, cols_d = dom // 9, (dom % 9) // 3, dom % 3
    form = ctx.pass_wpt(trunc, rows_d, cols_d, prec_d, N)
    kernel_share = {names.get(k, "class%d" % k): round(v["ms"] / max(1e-9, total_pass_ms), 4)
                    for k, v in stats.items() if v["launches"]}
    roofline = {"bound": "alu", "kernel": names.get(dom, "class%d" % dom),
                "form": "tiled (lanes = targets, TMA-staged sources)" if form == 1 else
                        ("chunk-balanced streaming (32-source chunks split evenly over the resident warps)"
                         if form == 3 else "streaming, %d warps per target" % form),
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None,
                "traffic_note": "DRAM bytes per launch are not counted in this run; they come from an ncu capture "
                                "of the same kernel (sources L1/L2-resident: a few hundred KB per launch)",
                "peak_source": ("FP32 CUDA-core peak %d SMs x 128 lanes x 2 x %.0f MHz (sm_max_mhz of %s "
                                "MEASURED_PEAKS.json)" % (sms, sm_max, peak_src)) if is_f32 else
                               "GB300 FP64 nominal 1.25 TFLOP/s",
                "flop_convention": "algorithmic flops of the pair formula (FMA = 2); double-float passes count "
                                   "the same formula although each flop costs ~10-20 FP32 instructions",
                "timing": "CUDA events around each of 40 back-to-back launches of this pass on the library stream "
                          "(same N, positions, tuned form), right after the timed region",
                "in_step_avg_launch_ms": in_step_ms, "in_step_frac": flops_per_launch / (in_step_ms * 1e-3) / 1e12 /
                peak, "profiled_ms_per_step": prof_ms / args.steps,
                "flops_per_launch": flops_per_launch, "avg_launch_ms": avg_ms, "time_share": kernel_share}

    # ---- end to end through the host-pointer C ABI (H2D + solve + D2H per step)
    h = gbi.h(trunc)
    pin = lambda shape: torch.zeros(shape, dtype=torch.float64).pin_memory()
    hR, hVa, hOa, hVH, hFe, hTe = (pin((N, 3)), pin((N, 3)), pin((N, 3)), pin((N, h)), pin((N, 3)), pin((N, 3)))
    hR.copy_(R0.cpu())
    hVa.copy_(inp["Va"].cpu())
    hOa.copy_(inp["Oa"].cpu())
    hVH.copy_(inp["VH"].cpu())
    hFe.copy_(inp["Fe"].cpu())
    hTe.copy_(inp["Te"].cpu())
    hV, hOm, hQH = pin((N, 3)), pin((N, 3)), pin((N, h))
    ptrs = [t.data_ptr() for t in (hR, hVa, hOa, hVH, hFe, hTe, hV, hOm, hQH)]
    for _ in range(2):
        ctx.solve_host_ptrs(prm, N, ptrs)
    barrier()
    e_pairs, e_t = 0, 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        info, _ = ctx.solve_host_ptrs(prm, N, ptrs)
        e_t += time.perf_counter() - t0
        e_pairs += info.pair_interactions
    barrier()
    h2d = 8 * N * (5 * 3 + h)
    d2h = 8 * N * (2 * 3 + h)
    e2e = {"value": e_pairs / e_t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "solves_per_s": args.steps / e_t, "call": "gbi_solve_host (pinned host buffers, one solve per step)",
           "start": "cold (zero initial guess) every call, the N=1024 initial suspension"}

    # ---- secondary: superposition trap pass at N = 10^4 (closed-form kernel, FP32)
    c3 = workloads.config3()
    R3 = torch.tensor(c3["R"], dtype=torch.float64, device=dev)
    p3 = torch.tensor(c3["p"], dtype=torch.float64, device=dev)
    in3 = ctx.trap_inputs(len(R3), 2, c3["k"], c3["vs"], c3["s0"], c3["d0"], R3, p3)
    prm3 = gbi.params(a=c3["a"], eta=c3["eta"], trunc=2, precision=1)
    V3 = torch.empty_like(R3)
    O3 = torch.empty_like(R3)
    for _ in range(3):
        ctx.superpose(prm3, R3, in3["Va"], in3["Oa"], in3["VH"], in3["Fe"], in3["Te"], V3, O3)
    ctx.set_profiling(True)
    barrier()
    ev0.record(stream)
    n3 = 20
    for _ in range(n3):
        ctx.superpose(prm3, R3, in3["Va"], in3["Oa"], in3["VH"], in3["Fe"], in3["Te"], V3, O3)
    ev1.record(stream)
    ev1.synchronize()
    t3 = ev0.elapsed_time(ev1) / 1e3
    s3 = ctx.kernel_stats(gbi._native.TRAP_F32)
    ctx.set_profiling(False)
    N3 = len(R3)
    ach3 = s3["flops"] / (s3["ms"] * 1e-3) / 1e12
    superposition = {"workload": c3["name"], "N": N3, "value": n3 * N3 * (N3 - 1) / t3, "unit": UNIT,
                     "ms_per_pass": 1e3 * t3 / n3,
                     "roofline": {"bound": "alu", "kernel": "trap superposition pass (pack + trap_pairs_f2 + finish)",
                                  "achieved": ach3, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach3 / fp32_peak,
                                  "traffic": None, "avg_launch_ms": s3["ms"] / max(1, s3["launches"])},
                     "note": "inputs resident (L2-sized), not flushed"}

    # ---- the same cloud above a plane no-slip wall (lowest centre at 2a): unbounded
    # superposition plus the wall's image flows (FP32)
    Rw = R3.clone()
    Rw[:, 2] += 2.0 * c3["a"] - Rw[:, 2].min()
    inw = ctx.trap_inputs(len(Rw), 2, c3["k"], c3["vs"], c3["s0"], c3["d0"], Rw, p3)
    for _ in range(2):
        ctx.wall_superpose(prm3, Rw, inw["Va"], inw["Oa"], inw["VH"], inw["Fe"], inw["Te"], V3, O3)
    ctx.set_profiling(True)
    ev0.record(stream)
    nw = 5
    for _ in range(nw):
        ctx.wall_superpose(prm3, Rw, inw["Va"], inw["Oa"], inw["VH"], inw["Fe"], inw["Te"], V3, O3)
    ev1.record(stream)
    ev1.synchronize()
    tw = ev0.elapsed_time(ev1) / 1e3
    sw = ctx.kernel_stats(gbi._native.WALL_F32)
    ctx.set_profiling(False)
    achw = sw["flops"] / (sw["ms"] * 1e-3) / 1e12
    wall_line = {"workload": c3["name"] + "_above_wall", "N": N3,
                 "value": nw * N3 * (N3 - 1) / tw, "unit": UNIT, "image_terms_per_s": nw * N3 * N3 / tw,
                 "ms_per_evaluation": 1e3 * tw / nw,
                 "roofline": {"bound": "alu",
                              "kernel": "wall images (records + k_wall_pairs<float>, nested dual numbers + reduce)",
                              "achieved": achw, "peak": fp32_peak, "unit": "TFLOP/s", "frac": achw / fp32_peak,
                              "flops_per_image_term": sw["flops"] / max(1, sw["launches"]) / (N3 * N3),
                              "traffic": None, "avg_launch_ms": sw["ms"] / max(1, sw["launches"])},
                 "note": "value counts the unbounded pairs N(N-1) per evaluation; the image terms are N^2 "
                         "(every sphere's own image included)"}

    # ---- periodic cube (point forces, Ewald sums): the chosen plan (particle mesh where it
    # pays) against the direct Ewald sum and every pair
    periodic_line = {}
    for Np in (10000, 100000):
        Lp = (Np * 4.0 * math.pi / 3.0 / 0.1) ** (1.0 / 3.0)        # volume fraction 0.1 of a = 1
        rng_p = __import__("numpy").random.default_rng(12345 + Np)
        Rp = torch.tensor(rng_p.uniform(0.0, Lp, size=(Np, 3)), dtype=torch.float64, device=dev)
        Fp = torch.tensor(rng_p.normal(size=(Np, 3)) * 0.1, dtype=torch.float64, device=dev)
        Vap = torch.zeros_like(Rp)
        res = {}
        for label, cells, mesh in (("chosen", 0, 0), ("direct_ewald", 0, -1), ("every_pair", -1, -1)):
            Vp, plan = ctx.periodic_superpose(prm3, Lp, Rp, Vap, Fp, cells=cells, mesh=mesh)
            reps = 3 if label == "chosen" else 1     # the O(N^2) / O(N^1.5) baselines run long
            ev0.record(stream)
            for _ in range(reps):
                ctx.periodic_superpose(prm3, Lp, Rp, Vap, Fp, Vp, cells=cells, mesh=mesh)
            ev1.record(stream)
            ev1.synchronize()
            res[label] = {"ms": ev0.elapsed_time(ev1) / reps, **plan}
            res[label + "_V"] = Vp.clone()
        Vref = res.pop("every_pair_V")
        scale = float(Vref.abs().max())
        for label in ("chosen", "direct_ewald"):
            res[label]["max_diff_over_max_V"] = float((res.pop(label + "_V") - Vref).abs().max()) / scale
        periodic_line["N%d" % Np] = {"L": Lp, **res,
                                     "speedup_of_chosen_over_every_pair": res["every_pair"]["ms"] / res["chosen"]["ms"]}
    periodic_line["note"] = ("FP32 Ewald sums in the periodic cube (Hasimoto's zero-mean-flow limit) at volume "
                             "fraction 0.1; chosen: the plan of the work estimate (cells per side and, where it "
                             "pays, the particle mesh: order-8 B-splines, K >= 5 xi L, ~N log N); direct_ewald: the "
                             "best split with direct wave-space sums (~N^1.5); every_pair: the minimum image over "
                             "all pairs (~N^2).  Differences are against every_pair, over the largest velocity.")

    # ---- flow field after the solve: a 64^3 grid through the N = 1024 suspension (FP32)
    V2, O2, Q2, _, _ = ctx.solve(prm, R0, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
    side = float(c["side"])
    g1 = torch.linspace(-side / 2, side / 2, 64, dtype=torch.float64, device=dev)
    Xg = torch.stack(torch.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3).contiguous()
    prmf = gbi.params(a=c["a"], eta=c["eta"], trunc=trunc, precision=1)
    Ug = torch.empty_like(Xg)
    ctx.flow(prmf, R0, inp["Fe"], inp["Te"], Q2, Xg, Ug)
    ctx.set_profiling(True)
    nfl = 5
    n_inside = 0
    for _ in range(nfl):
        _, n_inside = ctx.flow(prmf, R0, inp["Fe"], inp["Te"], Q2, Xg, Ug)
    sf = ctx.kernel_stats(gbi._native.FLOW_F32)
    ctx.set_profiling(False)
    fl_ms = sf["ms"] / max(1, sf["launches"])
    ach_f = sf["flops"] / (sf["ms"] * 1e-3) / 1e12
    flowline = {"points": int(Xg.shape[0]), "spheres": N, "trunc": trunc, "points_inside_spheres": n_inside,
                "ms_per_evaluation": fl_ms, "points_per_s": Xg.shape[0] / (fl_ms / 1e3),
                "point_sphere_terms_per_s": Xg.shape[0] * N / (fl_ms / 1e3),
                "roofline": {"bound": "alu", "kernel": "k_flow<l3, float> (1s rows of a zero-radius target)",
                             "achieved": ach_f, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach_f / fp32_peak,
                             "traffic": None},
                "grid": "64^3 points on the suspension's cube (side %.1f a)" % side}

    # ---- two squirmers in a trap: the frozen opposite pair and the orbits of other angles
    pair_orbits = squirmer_pair_orbits(ctx, gbi, dev, stream)

    # ---- trajectories: N = 64 FP64 re-solved steps; N = 10^4 superposition trap (10^4 steps)
    try:
        traj64 = trajectory_n64(ctx, gbi, dev, stream)
    except gbi.GbiError as e:
        traj64 = {"status": str(e)}
    traj3 = trajectory_trap(ctx, gbi, dev, stream, c3["R"], c3["p"], c3["k"], c3["steps"], c3["dt"])
    traj3.update({"workload": c3["name"], "initial": "Gaussian cloud sigma = 20a about the trap centre"})
    # the paper's geometry: 10^4 squirmers uniform on the sphere of radius R* = 1256.6a
    rng = np.random.default_rng(workloads.SEED_BASE + 33)
    u = rng.normal(size=(N3, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    Rp = 1256.6
    kp = 6 * math.pi * workloads.ETA_DEFAULT * 0.1 / Rp
    trajp = trajectory_trap(ctx, gbi, dev, stream, Rp * u, u.copy(), kp, 2000, c3["dt"])
    trajp.update({"workload": "N10000_trap_paper_geometry",
                  "initial": "uniform on the sphere of radius R* = 1256.6a, orientations radial",
                  "note": "short run (%.0f time units); the paper's snapshots reach 8 tau_r = %.3g time units"
                          % (2000 * c3["dt"], 8 * 8 * math.pi * workloads.ETA_DEFAULT / kp)})

    # ---- secondary: 256 independent suspensions (N log-uniform in [32, 4096]) in one batched solve
    c4 = workloads.config4()
    offs = [0]
    for sy in c4["systems"]:
        offs.append(offs[-1] + len(sy["R"]))
    R4 = torch.tensor(np.concatenate([sy["R"] for sy in c4["systems"]]), dtype=torch.float64, device=dev)
    p4 = torch.tensor(np.concatenate([sy["p"] for sy in c4["systems"]]), dtype=torch.float64, device=dev)
    in4 = ctx.trap_inputs(len(R4), 2, c4["k"], c4["vs"], c4["s0"], c4["d0"], R4, p4)
    prm4 = gbi.params(a=c4["a"], eta=c4["eta"], trunc=2, precision=args.precision, rtol=1e-10, restart=40,
                      inner_rtol=1e-5)
    tuned4 = ctx.tune(2, offs)
    for _ in range(2):
        ctx.batch_solve(prm4, offs, R4, in4["Va"], in4["Oa"], in4["VH"], in4["Fe"], in4["Te"])
    barrier()
    n4 = 3
    b_ms, b_pairs = 0.0, 0
    for _ in range(n4):
        flush.fill_(1.0)
        ev0.record(stream)
        _, _, _, i4, _ = ctx.batch_solve(prm4, offs, R4, in4["Va"], in4["Oa"], in4["VH"], in4["Fe"], in4["Te"])
        ev1.record(stream)
        ev1.synchronize()
        b_ms += ev0.elapsed_time(ev1)
        b_pairs += i4.pair_interactions
    # the config-4 step: trap inputs + batched solve + Euler update of all 256 systems, one
    # replayed CUDA graph per step once the call repeats
    R4s, p4s = R4.clone(), p4.clone()
    rep0 = ctx.solve_graph_replays()
    for _ in range(3):
        ctx.batch_trap_step(prm4, offs, R4s, p4s, 0.1, c4["k"], c4["vs"], c4["s0"], c4["d0"], False, 1)
    barrier()
    nst = 5
    st_ms, st_pairs = 0.0, 0
    rep1 = ctx.solve_graph_replays()
    for _ in range(nst):
        flush.fill_(1.0)
        ev0.record(stream)
        ist = ctx.batch_trap_step(prm4, offs, R4s, p4s, 0.1, c4["k"], c4["vs"], c4["s0"], c4["d0"], False, 1)
        ev1.record(stream)
        ev1.synchronize()
        st_ms += ev0.elapsed_time(ev1)
        st_pairs += ist.pair_interactions
    graph_steps = ctx.solve_graph_replays() - rep1
    # its dominant pass class, event-timed per launch inside one more batched solve
    ctx.set_profiling(True)
    ctx.batch_solve(prm4, offs, R4, in4["Va"], in4["Oa"], in4["VH"], in4["Fe"], in4["Te"])
    st4 = {cls: ctx.kernel_stats(cls) for cls in range(gbi._native.N_KERNEL_CLASSES)}
    ctx.set_profiling(False)
    dom4 = max(st4, key=lambda k: st4[k]["ms"])
    ach4 = st4[dom4]["flops"] / (st4[dom4]["ms"] * 1e-3) / 1e12
    batched = {"workload": c4["name"], "systems": len(c4["systems"]), "spheres": len(R4), "trunc": 2,
               "value": b_pairs / (b_ms / 1e3), "unit": UNIT, "ms_per_batch_solve": b_ms / n4,
               "systems_per_s": n4 * len(c4["systems"]) / (b_ms / 1e3), "lockstep_iters": i4.iters,
               "rel_residual": i4.rel_residual, "tuned_wpt": dict(zip(TUNED_PASSES, tuned4)),
               "step": {"call": "gbi_batch_trap_step (trap inputs + batched solve + Euler update, all systems)",
                        "ms_per_step": st_ms / nst, "value": st_pairs / (st_ms / 1e3), "unit": UNIT,
                        "steps_timed": nst, "steps_replayed_as_one_graph": graph_steps,
                        "systems_per_s": nst * len(c4["systems"]) / (st_ms / 1e3)},
               "roofline": {"bound": "alu", "kernel": names.get(dom4, "class%d" % dom4).replace("l%d" % trunc, "l2"),
                            "achieved": ach4, "peak": fp32_peak if (9 <= dom4 < 27) else FP64_NOMINAL_TFLOPS,
                            "unit": "TFLOP/s",
                            "frac": ach4 / (fp32_peak if (9 <= dom4 < 27) else FP64_NOMINAL_TFLOPS),
                            "traffic": None, "avg_launch_ms": st4[dom4]["ms"] / max(1, st4[dom4]["launches"]),
                            "timing": "CUDA events around every pass of one batched solve (direct launches)"}}

    # ---- secondary: learned near-field correction (training, errors, N = 10^5 evaluation)
    learned = learned_nearfield(ctx, gbi, dev, stream, load_peaks()[0])

    if rank == 0:
        # ---- CPU baseline: the oracle on bounded samples, this machine's cores
        cpu = oracle_baselines(workloads.config1(), c, c3)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "precision": modes["p%d" % args.precision]["precision"] + "; FP64 Arnoldi/Givens",
                "data": "synthetic",
                "config": {"workload": c["name"], "N": N, "trunc": trunc, "h": h, "volume_fraction": 0.05,
                           "min_sep_a": 2.5, "overlap_guard_a": 2.0, "rtol": 1e-10, "restart": 40,
                           "inner_rtol": 1e-5,
                           "step": "trap inputs + full Galerkin solve + Euler update",
                           "trajectory": "from the initial suspension, reset to it every %d steps" % RESET_EVERY,
                           "l2": "flushed (256 MB write) before every timed step",
                           "parallelism": "replicas" if world > 1 else "single GPU", "sms": sms},
                "solves_per_s": solves_per_s, "residual_vs_fp64_system": err["residual_vs_fp64_system"],
                "error_vs_fp64": err, "vs_fp64_gmres": vs_fp64, "precision_modes": modes,
                "per_step": {"gmres_iters": step_stats["iters"] / args.steps,
                             "refinements": step_stats["refinements"] / args.steps,
                             "fp32_passes": step_stats["matvecs_f32"] / args.steps,
                             "high_precision_passes": step_stats["matvecs_hp"] / args.steps,
                             "max_rel_residual": step_stats["max_residual"],
                             "start": "cold (zero initial guess) every step: mixed precision"},
                "roofline": roofline,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
                "superposition": superposition, "wall_superposition": wall_line,
                "periodic_superposition": periodic_line, "flow_field": flowline, "config1_trajectory": traj64, "config3_trajectory": traj3,
                "config3_paper_geometry": trajp, "squirmer_pair_orbits": pair_orbits, "batched": batched, "learned_nearfield": learned,
                "tuned_wpt": dict(zip(TUNED_PASSES, tuned))}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=3, choices=[0, 1, 2, 3],
                    help="0 all FP64; 1 FP32 GMRES + FP64 refinement; 2 FP32 GMRES + double-float refinement, "
                         "RHS and outputs; 3 as 2 with FP32 RHS and outputs")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
