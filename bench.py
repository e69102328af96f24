#!/usr/bin/env python
"""Benchmark of the Galerkin boundary-integral hot path on GB300.

Workload (default): N = 1024 active spheres at volume fraction 0.05, truncation
l <= 3 (25 higher components per sphere), harmonic trap k = 0.01, V^a = 0.1 p,
V^(2s) = 0.05 (pp - I/3).  One step = trap inputs from (R, p), the full
traction solve (FP64 right-hand-side pass, restarted GMRES with FP32 pair sums
and FP64 Arnoldi, FP64 iterative refinement to ||b - A q|| / ||b|| <= 1e-10,
FP64 output pass) and one forward-Euler update, all inside libgbi.

Metric: pair-interactions/s (ordered pairs summed over every pair pass of the
step) and solves/s.  Also reported: the roofline of the dominant kernel (event
timed live in the timed region), the end-to-end number through the host-pointer
C-ABI call, the N = 10^4 superposition pass, and the FP64 CPU oracle timed on
a bounded sample on this machine's cores.

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
SMS, FP32_LANES = 152, 128


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_alu_peak_tflops(sm_mhz):
    return SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12


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
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# passes timed by gbi_tune, in the order of its result
TUNED_PASSES = ["HH_f32", "HH_df", "HL_df", "Lall_df", "HL_f32", "Lall_f32"]
RESET_EVERY = 20     # timed trap steps between returns to the initial suspension
# DRAM bytes (read + write) per launch of a pass class on this workload, from an ncu capture
# of the current kernel (profiles/pair_stream_kernel_l3_HH_f32_N1024.md, 1024 targets, l <= 3):
# class 17 = FP32 rows H / columns H.  Reported as roofline.traffic when that class dominates.
NCU_TRAFFIC_BYTES = {17: 168704}


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
    return {"workload": c5["name"], "N": N5, "value": pairs5 / (ms_full / 1e3), "unit": UNIT,
            "ms_per_evaluation": ms_full, "network_pairs": P,
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
    # a non-default stream lets the library replay its Arnoldi chunks from CUDA graphs
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

    # ---- pair-kernel tuning (warps per target of each pass), outside the timed region
    tuned = ctx.tune(trunc, [0, N])

    # ---- accuracy statement (outside the timed region): mixed vs all-FP64 on the GPU
    inp = ctx.trap_inputs(N, trunc, c["k"], c["vs"], c["s0"], c["d0"], R0, p0)
    V1, O1, Q1, i1, _ = ctx.solve(prm, R0, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
    prm64 = gbi.params(a=c["a"], eta=c["eta"], trunc=trunc, precision=0, rtol=1e-10, restart=40)
    V0, O0, Q0, i0, _ = ctx.solve(prm64, R0, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
    torch.cuda.synchronize(dev)

    def rel(a, b):
        return float((a - b).abs().max() / b.abs().max())

    def rel_rows(a, b):   # max_n |a_n - b_n| / max_n |b_n| (per-sphere 2-norms)
        return float((a - b).norm(dim=1).max() / b.norm(dim=1).max())
    err = {"V_rel": rel(V1, V0), "Omega_rel": rel(O1, O0), "QH_rel": rel(Q1, Q0),
           "V_rel_per_particle": rel_rows(V1, V0), "Omega_rel_per_particle": rel_rows(O1, O0),
           "QH_rel_per_mode": {name: rel(Q1[:, o:o + k], Q0[:, o:o + k]) for name, o, k in h_mode_slices(trunc)},
           "mixed_residual": i1.rel_residual, "fp64_residual": i0.rel_residual,
           "mixed_iters": i1.iters, "mixed_refinements": i1.refinements, "fp64_iters": i0.iters}

    # ---- the same solve in plain FP64 GMRES (precision 0) against the mixed form: solves/s
    # on this GPU at the same tolerance, the mixed V within V_rel of the FP64 one (outside
    # the timed region; CUDA events on the library stream, each solve after an L2 flush)
    sv0, sv1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def solve_ms(pr, reps):
        tot = 0.0
        for _ in range(reps):
            flush.fill_(1.0)
            sv0.record(stream)
            ctx.solve(pr, R0, inp["Va"], inp["Oa"], inp["VH"], inp["Fe"], inp["Te"])
            sv1.record(stream)
            sv1.synchronize()
            tot += sv0.elapsed_time(sv1)
        return tot / reps
    ms64 = solve_ms(prm64, 3)
    ms_mixed = solve_ms(prm, 10)
    vs_fp64 = {"fp64_solves_per_s": 1e3 / ms64, "mixed_solves_per_s": 1e3 / ms_mixed,
               "fp64_ms_per_solve": ms64, "mixed_ms_per_solve": ms_mixed, "speedup": ms64 / ms_mixed,
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
    # ---- the same steps again with CUDA events around every pair pass (direct launches)
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

    # ---- dominant kernel and its roofline
    peaks, peak_src = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    tname = {0: "double", 1: "float", 2: "double-float"}
    sname = {0: "all", 1: "L", 2: "H"}
    names = {pr * 9 + r * 3 + cc: "pair_kernel<l3, %s, %s, %s>" % (sname[r], sname[cc], tname[pr])
             for pr in range(3) for r in range(3) for cc in range(3)}
    names[27] = "trap pass FP64"
    names[28] = "trap pass FP32"
    dom = max(stats, key=lambda k: stats[k]["ms"])
    st = stats[dom]
    avg_ms = st["ms"] / max(1, st["launches"])
    flops_per_launch = st["flops"] / max(1, st["launches"])
    achieved = flops_per_launch / (avg_ms * 1e-3) / 1e12
    is_f32 = dom == 28 or (9 <= dom < 27)       # FP32 and double-float classes run on the FP32 pipe
    peak = fp32_alu_peak_tflops(sm_max) if is_f32 else FP64_NOMINAL_TFLOPS
    kernel_share = {names.get(k, "class%d" % k): round(v["ms"] / max(1e-9, sum(s["ms"] for s in stats.values())), 4)
                    for k, v in stats.items() if v["launches"]}
    roofline = {"bound": "alu", "kernel": names.get(dom, "class%d" % dom), "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": NCU_TRAFFIC_BYTES.get(dom),
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum, "
                                "profiles/pair_stream_kernel_l3_HH_f32_N1024.md)",
                "peak_source": ("FP32 CUDA-core peak 152 SMs x 128 lanes x 2 x %.0f MHz (sm_max_mhz of %s "
                                "MEASURED_PEAKS.json)" % (sm_max, peak_src)) if is_f32 else
                               "GB300 FP64 nominal 1.25 TFLOP/s",
                "flop_convention": "algorithmic flops of the pair formula (FMA = 2); double-float passes count "
                                   "the same formula although each flop costs ~10-20 FP32 instructions",
                "timing": "CUDA events around every pair pass on the library stream, in a replay of the same "
                          "steps right after the timed region (per-pass events need direct launches; the timed "
                          "region replays Arnoldi chunks from CUDA graphs)",
                "profiled_ms_per_step": prof_ms / args.steps,
                "flops_per_launch": flops_per_launch, "avg_launch_ms": avg_ms, "launches": st["launches"],
                "time_share": kernel_share}

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
                     "roofline": {"bound": "alu", "kernel": "trap superposition pass (pack + trap_pairs<float> + finish)", "achieved": ach3,
                                  "peak": fp32_alu_peak_tflops(sm_max), "unit": "TFLOP/s",
                                  "frac": ach3 / fp32_alu_peak_tflops(sm_max), "traffic": None,
                                  "avg_launch_ms": s3["ms"] / max(1, s3["launches"])},
                     "note": "inputs resident (L2-sized), not flushed"}

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
    batched = {"workload": c4["name"], "systems": len(c4["systems"]), "spheres": len(R4), "trunc": 2,
               "value": b_pairs / (b_ms / 1e3), "unit": UNIT, "ms_per_batch_solve": b_ms / n4,
               "systems_per_s": n4 * len(c4["systems"]) / (b_ms / 1e3), "lockstep_iters": i4.iters,
               "rel_residual": i4.rel_residual, "tuned_wpt": dict(zip(TUNED_PASSES, tuned4))}

    # ---- secondary: learned near-field correction (training, errors, N = 10^5 evaluation)
    learned = learned_nearfield(ctx, gbi, dev, stream, load_peaks()[0])

    if rank == 0:
        # ---- CPU baseline: the oracle on a bounded sample, this machine's cores
        rate, dtc = oracle_pair_rate(c["R"], trunc, c["a"], 12000)
        cpu = {"value": rate, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
               "sample": "12000 random ordered pairs of the N=1024 l<=3 suspension, dense FP64 31x31 pair "
                         "blocks + apply (%.1f s)" % dtc}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "precision": {0: "FP64 throughout", 1: "FP32 pair sums in GMRES; FP64 RHS, residuals, outputs; FP64 "
                              "Arnoldi/Givens", 2: "FP32 pair sums in GMRES; double-float (FP32-pipe, ~48-bit) RHS, "
                              "residuals, outputs; FP64 Arnoldi/Givens",
                              3: "FP32 pair sums in GMRES, RHS and outputs; double-float refinement residuals; "
                              "FP64 Arnoldi/Givens"}[args.precision],
                "data": "synthetic",
                "config": {"workload": c["name"], "N": N, "trunc": trunc, "h": h, "volume_fraction": 0.05,
                           "min_sep_a": 2.5, "overlap_guard_a": 2.0, "rtol": 1e-10, "restart": 40,
                           "inner_rtol": 1e-5,
                           "step": "trap inputs + full Galerkin solve + Euler update",
                           "trajectory": "from the initial suspension, reset to it every %d steps" % RESET_EVERY,
                           "l2": "flushed (256 MB write) before every timed step",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "solves_per_s": solves_per_s, "error_vs_fp64": err, "vs_fp64_gmres": vs_fp64,
                "per_step": {"gmres_iters": step_stats["iters"] / args.steps,
                             "refinements": step_stats["refinements"] / args.steps,
                             "fp32_passes": step_stats["matvecs_f32"] / args.steps,
                             "high_precision_passes": step_stats["matvecs_hp"] / args.steps,
                             "max_rel_residual": step_stats["max_residual"],
                             "start": "cold (zero initial guess) every step: mixed precision"},
                "roofline": roofline,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": launches,
                "superposition": superposition, "batched": batched, "learned_nearfield": learned,
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
