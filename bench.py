#!/usr/bin/env python3
"""Benchmark of the LSG-CPD E-step / EM engine on GB300.

A step = one full registration of the RGBD-shaped pair (20,000 x 20,000 points,
synthetic room ray-cast from a 160 x 125 pinhole camera): preprocessing (kNN,
normals, surface variation, penalties), initialisation and 50 EM iterations
(fused E step + FP64 moment combine + FP64 Newton M step), through the C ABI.

value = E-step pair evaluations per second (50 x N x M per step) with the
inputs resident in HBM; e2e = the same metric through the same C call with
pinned host inputs (H2D inside the call, result read back to the host).
The roofline object reports the hot E-step kernel, timed live with CUDA events
on the stream it is launched on, against the FP32-pipe peak (ALU bound).

Other workloads (--workload): sphere1k (1,000 x 1,000 sphere + plane), lidar100k
(two 64 x 1,563 LiDAR scans), superquadric500k (500,000 x 500,000 range scan),
each one full registration per step like the default.
With --workload batch256 a step is instead one batched registration of 256
independent pairs with N, M log-uniform in [500, 20,000] (one launch per stage
for the whole batch); the line then also carries the same 256 pairs registered
one after another through lsgcpd_register (the plain per-pair form).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload rgbd20k|sphere1k|lidar100k|superquadric500k|batch256]
                       [--precision 0|1|2] [--iters I] [--no-cpu-baseline]
Under torchrun every rank registers its own independent pair (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "E-step pair-evals/sec & EM iters/sec at 1 GB300; % FP32/SFU roofline; rot err vs FP64"
UNIT = "pair-evals/s"
FLOPS_PER_PAIR = 27  # FP32-pipe operations per (source, target) pair, the fixed algorithmic count
TC_FP32_OPS_PER_PAIR = 11  # what stays on the FP32 pipe when the moment sums run on the tensor cores
EX2_PER_PAIR = 1
SM_MAX_MHZ_NOMINAL = 2070.0
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--iters", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["rgbd20k", "sphere1k", "lidar100k", "superquadric500k", "batch256"],
                    default="rgbd20k")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the second measurement of the same workload with precision 2")
    ap.add_argument("--precision", type=int, choices=[0, 1, 2], default=0,
                    help="0: FP32 E step; 1: f16x2 exponentials (mixed precision); "
                         "2: TF32 exponentials with the moment sums on the tensor cores")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(offset, rank):
    """Seed of rank `rank`'s independent problem (weak scaling: every rank its own pair)."""
    from paper_2103_15039_gb300 import synth
    return synth.SEED_BASE + offset + 1000 * rank


def reduce_max(values, ws, device):
    """Max over ranks of per-rank times (the job is as slow as its slowest rank)."""
    if ws == 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_throughput(units_per_rank, ws, ms):
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return ws * units_per_rank / (ms / 1e3)


# single-pair workloads: name -> (seed offset, generator name, label)
SINGLE = {
    "sphere1k": (1, "sphere_plane_pair", "sphere_plane_1000x1000"),
    "rgbd20k": (2, "rgbd_room_pair", "rgbd_room_20000x20000"),
    "lidar100k": (3, "lidar_pair", "lidar_64x1563_100032x100032"),
    "superquadric500k": (5, "superquadric_pair", "superquadrics_500000x500000"),
}


def workload(rank, name="rgbd20k"):
    from paper_2103_15039_gb300 import synth
    off, gen, _ = SINGLE[name]
    seed = rank_seed(off, rank)
    c = getattr(synth, gen)(seed=seed)
    return c, seed


def batch_workload(rank):
    import numpy as np

    from paper_2103_15039_gb300 import synth
    seed = rank_seed(4, rank)
    pairs = synth.batch_pairs(seed=seed)
    X = np.concatenate([q["X"] for q in pairs]).astype(np.float32)
    Y = np.concatenate([q["Y"] for q in pairs]).astype(np.float32)
    n_off = np.concatenate([[0], np.cumsum([len(q["X"]) for q in pairs])]).astype(np.int64)
    m_off = np.concatenate([[0], np.cumsum([len(q["Y"]) for q in pairs])]).astype(np.int64)
    return pairs, X, n_off, Y, m_off, seed


E_STEP_DESC = {0: "fp32 (packed f32x2) + ex2.approx",
               1: "fp32 residuals + f16x2 ex2.approx",
               2: "fp32 residuals + ex2.approx, exponentials truncated to tf32, moment sums on tcgen05 "
                  "(tf32 x hi/lo features, f32 accumulation in tensor memory)"}
DTYPE = {0: "f32", 1: "f32+f16", 2: "f32+tf32"}
# workloads whose line also times the f16x2-exponential path and its error against FP32
HALF2_WORKLOADS = ("lidar100k", "superquadric500k")


def config_obj(c, seed, iters, n_gpus, precision=0, name="rgbd20k"):
    extra = {"overlap": round(float(c["overlap"]), 4)} if "overlap" in c else {}
    return {"workload": SINGLE[name][2], "N": int(len(c["X"])), "M": int(len(c["Y"])),
            "em_iters": iters, "knn_k": 10, "w": 0.1, "alpha_max": 2.0, "lambda": 0.2, "seed": seed,
            **extra,
            "e_step": E_STEP_DESC[precision],
            "m_step": "double-float Newton (FP32 pairs) on FP64 moments", "l2": "flushed between steps (256 MiB write)",
            "parallelism": f"replicas x{n_gpus} (independent pairs per GPU)"}


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

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
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


def kernel_source_hash(precision=0):
    """sha256 over the sources that define the E-step kernel (its file and its copy pipeline)."""
    h = hashlib.sha256()
    for name in (("estep_tc.cu",) if precision >= 2 else ("estep.cu",)) + ("estep_common.cuh", "pipeline.cuh"):
        with open(os.path.join(ROOT, "paper_2103_15039_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def profile_traffic(precision=0, workload="rgbd20k"):
    """DRAM traffic per E-step launch from the committed ncu summary, if it was taken
    on the current kernel source and on this workload (null otherwise)."""
    if workload != "rgbd20k" or precision not in (0, 2):
        return None
    name = "estep_tc_rgbd20k_traffic.json" if precision == 2 else "estep_rgbd20k_traffic.json"
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            prof = json.load(f)
        h = kernel_source_hash(precision)
    except OSError:
        return None
    if prof.get("estep_source_sha256") != h:
        return None
    return prof.get("dram_bytes_per_launch")


def settle(step, seconds=2.0):
    """Untimed work before the warm-up steps, so that the GPU's clocks have settled
    (a fresh box runs its first second or so a few percent slower)."""
    import torch
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        step()
        torch.cuda.synchronize()


def plan_obj(ctx):
    """The E-step plan of the last call (sources per thread chosen by the autotuner)."""
    info = ctx.plan_info()
    return {"sources_per_thread": info["sources_per_thread"], "block": info["block"], "ctas": info["ctas"],
            "autotuned": info["tuned"], "tune_ms": {str(k): round(v, 5) for k, v in info["tune_ms"].items()}}


def cpu_baseline(c, got, iters, budget_s=40.0):
    """The FP64 oracle timed on this host's cores on the same pair.

    If the whole registration fits the budget (estimated from one E step on a
    subset of sources) it is run in full, which also gives the rotation and
    translation error of the GPU result against FP64; otherwise a bounded
    subset of one E step is timed."""
    import numpy as np

    import oracle
    X, Y = c["X"], c["Y"]
    N, M = len(X), len(Y)
    cores = os.cpu_count() or 1
    pre = oracle.preprocess(Y, 10, 2.0, 0.2)
    V, diag = oracle.volume(Y)
    ns = min(N, 2000)
    t0 = time.perf_counter()
    oracle.estep(X[:ns], Y, pre["normals"], pre["alpha"], np.eye(3), np.zeros(3), 0.05, 0.1, V)
    dt = time.perf_counter() - t0
    rate = ns * M / dt
    est_full = iters * N * M / rate
    out = {"unit": UNIT, "cores": cores, "kind": "oracle", "cpu": oracle.cpu_model()}
    if est_full <= budget_s:
        t0 = time.perf_counter()
        ref = oracle.register(X, Y, max_iters=iters)
        dt = time.perf_counter() - t0
        out["value"] = ref["iters"] * N * M / dt
        out["sample"] = f"full registration: kNN + geometry + {ref['iters']} EM iterations of the same pair"
        out["seconds"] = round(dt, 2)
        return out, dict(ref, diag=diag)
    ns = max(1, min(N, int(20.0 * rate / M)))
    t0 = time.perf_counter()
    oracle.estep(X[:ns], Y, pre["normals"], pre["alpha"], np.eye(3), np.zeros(3), 0.05, 0.1, V)
    dt = time.perf_counter() - t0
    out["value"] = ns * M / dt
    out["sample"] = f"one E step over {ns} of {N} sources x {M} targets"
    out["seconds"] = round(dt, 2)
    return out, None


def rotation_angle(Ra, Rb):
    """Angle of the relative rotation Ra^T Rb, 2 asin(|Ra - Rb|_F / (2 sqrt 2)) (accurate for small angles)."""
    import numpy as np
    d = np.linalg.norm(np.asarray(Ra, dtype=np.float64) - np.asarray(Rb, dtype=np.float64))
    return float(2.0 * np.arcsin(min(1.0, d / (2.0 * np.sqrt(2.0)))))


def errors_vs(got, ref, diag):
    """Rotation / translation / sigma^2 error of a GPU result against a reference result."""
    import numpy as np

    return {"rot_err_rad": rotation_angle(got["R"], ref["R"]),
            "trans_err_rel_diag": float(np.linalg.norm(got["t"] - ref["t"]) / diag),
            "sigma2_rel": abs(got["sigma2"] - ref["sigma2"]) / ref["sigma2"]}


def time_registrations(ctx, Xd, Yd, p, steps, flush, stream):
    """Device-resident registrations timed with CUDA events (L2 flushed before each): the step
    time without the library's per-kernel events, then the E step's per-launch time from a
    pass with them."""
    import torch

    def run(timing):
        ctx.set_timing(timing)
        ctx.register(Xd, Yd, p)
        step_ms, estep_ms, got = [], [], None
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            got = ctx.register(Xd, Yd, p)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            if timing:
                estep_ms.append(ctx.last_timing()["ms_estep"])
        return got, step_ms, estep_ms

    got, step_ms, _ = run(False)
    _, _, estep_ms = run(True)
    ctx.set_timing(False)
    return got, statistics.mean(step_ms), statistics.mean(estep_ms) / got["iters"]


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2103_15039_gb300 import binding

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    c, seed = workload(rank, args.workload)
    N, M = len(c["X"]), len(c["Y"])
    iters = args.iters
    ctx = binding.Context(local, N, M)
    p = binding.default_params(max_iters=iters, precision=args.precision)
    Xd = torch.from_numpy(c["X"]).cuda()
    Yd = torch.from_numpy(c["Y"]).cuda()
    Xh = torch.from_numpy(c["X"]).pin_memory()
    Yh = torch.from_numpy(c["Y"]).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # The library's per-kernel CUDA events are event nodes in the captured EM graph (four per
    # iteration, a few microseconds each), so the headline pass runs without them and a second
    # timed pass with them gives the E step's per-launch time and the device breakdown.
    ctx.set_timing(False)
    settle(lambda: ctx.register(Xd, Yd, p))
    for _ in range(max(args.warmup, 0)):
        got = ctx.register(Xd, Yd, p)
        ctx.register(Xh, Yh, p)

    # --- device-resident timed region (the headline) ---
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, launches = [], 0
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        got = ctx.register(Xd, Yd, p)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        launches += ctx.last_timing()["launches"]
    barrier()
    clk = clocks.stop()
    iters_run = got["iters"]

    # --- kernel-timing pass: the same steps with the library's per-kernel events ---
    ctx.set_timing(True)
    for _ in range(max(args.warmup, 1)):
        ctx.register(Xd, Yd, p)
    barrier()
    estep_ms, timed_step_ms = [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.register(Xd, Yd, p)
        e1.record(stream)
        e1.synchronize()
        timed_step_ms.append(e0.elapsed_time(e1))
        tm = ctx.last_timing()
        estep_ms.append(tm["ms_estep"])
    barrier()
    ctx.set_timing(False)
    # device-time breakdown of the last step of that pass (CUDA events recorded by the library)
    breakdown = {k: round(tm[k], 4) for k in ("ms_total", "ms_prep", "ms_estep", "ms_combine", "ms_mstep")}
    breakdown["ms_per_step_with_kernel_events"] = round(statistics.mean(timed_step_ms), 4)

    # --- end-to-end: pinned host inputs, copies inside the C call, result on the host ---
    e2e_s = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ctx.register(Xh, Yh, p)
        e2e_s.append(time.perf_counter() - t0)
    xfer = ctx.last_timing()
    assert np.allclose(r["R"], got["R"]) and np.allclose(r["t"], got["t"])

    ms, e2e_ms = reduce_max([statistics.mean(step_ms), statistics.mean(e2e_s) * 1e3], ws, "cuda")
    pairs_per_step = iters_run * N * M
    value = job_throughput(pairs_per_step, ws, ms)
    e2e_value = job_throughput(pairs_per_step, ws, e2e_ms)

    # roofline of the hot kernel (E step): per-launch time measured live
    t_launch = statistics.mean(estep_ms) / iters_run / 1e3
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12  # FP32-pipe Top/s
    # (per-launch time from the kernel-timing pass, on the stream the kernel runs on)
    # the tensor-core variant is measured against the FP32-pipe work it keeps (the moment sums
    # run on tcgen05 at ~11 % of the tensor pipe)
    ops = TC_FP32_OPS_PER_PAIR if args.precision == 2 else FLOPS_PER_PAIR
    achieved = ops * N * M / t_launch / 1e12
    ex2_rate = EX2_PER_PAIR * N * M / t_launch
    roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "traffic": profile_traffic(args.precision, args.workload),
            "kernel": "estep_tc_kernel" if args.precision >= 2 else "estep_kernel",
            "ms_per_launch": round(t_launch * 1e3, 5),
            "launch_timing": "CUDA events around every E-step launch, recorded as nodes of the captured EM graph "
                             "on its stream, in a second timed pass (the headline pass runs without them)",
            "pairs_per_s_per_launch": N * M / t_launch,
            "counted": f"{ops} FP32-pipe ops + {EX2_PER_PAIR} EX2 per pair, N*M pairs per launch",
            "peak_from": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {SM_MAX_MHZ_NOMINAL:.0f} MHz (max SM clock)",
            "ex2_per_s": ex2_rate}
    if clk.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = round(achieved / (sms * FP32_LANES_PER_SM * clk["sm_mhz"] * 1e6 / 1e12), 4)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
           "config": config_obj(c, seed, iters, ws, args.precision, args.workload),
           "em_iters_per_s": ws * iters_run / (ms / 1e3),
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": xfer["h2d_bytes"],
                   "d2h_bytes_per_step": xfer["d2h_bytes"], "ms_per_step": round(e2e_ms, 4),
                   "clock": "host wall"},
           "roofline": roof, "clocks": clk, "gpu_launches": launches,
           "mode": got["mode"], "iters_run": iters_run, "e_step_plan": plan_obj(ctx), "device_ms": breakdown}
    # the same workload with the moment sums on the tensor cores (precision 2), same protocol
    mixed = None
    if args.precision == 0 and not args.no_variants:
        p2 = binding.default_params(max_iters=iters, precision=2)
        for _ in range(max(args.warmup, 1)):
            ctx.register(Xd, Yd, p2)
        barrier()
        got2, ms2, est2 = time_registrations(ctx, Xd, Yd, p2, args.steps, flush, stream)
        barrier()
        diag = float(np.linalg.norm(c["Y"].max(0).astype(np.float64) - c["Y"].min(0).astype(np.float64)))
        mixed = {"precision": 2, "e_step": E_STEP_DESC[2], "dtype": DTYPE[2],
                 "value": job_throughput(got2["iters"] * N * M, ws, ms2), "unit": UNIT, "ms_per_step": round(ms2, 4),
                 "estep_ms_per_launch": round(est2, 5), "speedup_vs_fp32_step": round(ms / ms2, 4),
                 "speedup_vs_fp32_estep": round(t_launch * 1e3 / est2, 4),
                 "roofline": {"bound": "alu", "kernel": "estep_tc_kernel",
                              "achieved": round(TC_FP32_OPS_PER_PAIR * N * M / (est2 / 1e3) / 1e12, 3),
                              "peak": round(peak, 3), "unit": "TFLOP/s",
                              "frac": round(TC_FP32_OPS_PER_PAIR * N * M / (est2 / 1e3) / 1e12 / peak, 4),
                              "traffic": profile_traffic(2, args.workload),
                              "counted": f"{TC_FP32_OPS_PER_PAIR} FP32-pipe ops + 1 EX2 per pair (the moment "
                                         "sums run on tcgen05)"},
                 "iters_run": got2["iters"],
                 "vs_fp32_result": errors_vs(got2, got, diag)}
        out["mixed_precision"] = mixed
    # the range-scan workloads also compare the f16x2-exponential path (precision 1) with FP32
    half = None
    if args.precision == 0 and not args.no_variants and args.workload in HALF2_WORKLOADS:
        p1 = binding.default_params(max_iters=iters, precision=1)
        for _ in range(max(args.warmup, 1)):
            ctx.register(Xd, Yd, p1)
        barrier()
        got1, ms1, est1 = time_registrations(ctx, Xd, Yd, p1, args.steps, flush, stream)
        barrier()
        diag = float(np.linalg.norm(c["Y"].max(0).astype(np.float64) - c["Y"].min(0).astype(np.float64)))
        half = {"precision": 1, "e_step": E_STEP_DESC[1], "dtype": DTYPE[1],
                "value": job_throughput(got1["iters"] * N * M, ws, ms1), "unit": UNIT, "ms_per_step": round(ms1, 4),
                "estep_ms_per_launch": round(est1, 5), "speedup_vs_fp32_step": round(ms / ms1, 4),
                "iters_run": got1["iters"], "vs_fp32_result": errors_vs(got1, got, diag)}
        out["half2"] = half
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb, ref = cpu_baseline(c, got, iters_run)
        out["cpu_baseline"] = cb
        if ref:
            out["vs_fp64_oracle"] = errors_vs(got, ref, ref["diag"])
            if mixed:
                mixed["vs_fp64_oracle"] = errors_vs(got2, ref, ref["diag"])
        elif half and args.workload == "lidar100k":
            # the full FP64 registration does not fit the budget: both precisions against the
            # oracle over the first two EM iterations (about half a minute on 16 cores)
            import oracle
            ref2 = oracle.register(c["X"], c["Y"], max_iters=2)
            diag = float(np.linalg.norm(c["Y"].max(0).astype(np.float64) - c["Y"].min(0).astype(np.float64)))
            short = {}
            for prec, key in ((0, "fp32"), (1, "half2")):
                g2 = ctx.register(Xd, Yd, binding.default_params(max_iters=2, precision=prec))
                short[key] = errors_vs(g2, ref2, diag)
            out["vs_fp64_oracle_2_iterations"] = short
    ctx.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_batch(args):
    """A step = one lsgcpd_register_batch call over 256 uneven pairs."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2103_15039_gb300 import binding

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pairs, X, n_off, Y, m_off, seed = batch_workload(rank)
    P = len(pairs)
    Ns, Ms = np.diff(n_off), np.diff(m_off)
    nm = (Ns * Ms).astype(np.float64)
    iters = args.iters
    ctx = binding.Context(local, int(Ns.max()), int(Ms.max()))
    p = binding.default_params(max_iters=iters, precision=args.precision)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    Xh, Yh = torch.from_numpy(X).pin_memory(), torch.from_numpy(Y).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # headline pass without the library's per-kernel events (graph event nodes cost a few
    # microseconds each), then a kernel-timing pass with them for the roofline
    ctx.set_timing(False)
    settle(lambda: ctx.register_batch(Xd, n_off, Yd, m_off, p))
    for _ in range(max(args.warmup, 0)):
        got = ctx.register_batch(Xd, n_off, Yd, m_off, p)
        ctx.register_batch(Xh, n_off, Yh, m_off, p)
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, launches = [], 0
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        got = ctx.register_batch(Xd, n_off, Yd, m_off, p)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        launches += ctx.last_timing()["launches"]
    barrier()
    clk = clocks.stop()
    ctx.set_timing(True)
    ctx.register_batch(Xd, n_off, Yd, m_off, p)
    barrier()
    estep_ms = []
    for _ in range(args.steps):
        flush.zero_()
        ctx.register_batch(Xd, n_off, Yd, m_off, p)
        torch.cuda.synchronize()
        tm = ctx.last_timing()
        estep_ms.append(tm["ms_estep"])
    barrier()
    ctx.set_timing(False)
    plan = plan_obj(ctx)
    iters_run = int(got["iters"].max())
    pairs_per_step = float((got["iters"].astype(np.float64) * nm).sum())

    e2e_s = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = ctx.register_batch(Xh, n_off, Yh, m_off, p)
        e2e_s.append(time.perf_counter() - t0)
    xfer = ctx.last_timing()
    assert np.allclose(r["R"], got["R"]) and np.allclose(r["t"], got["t"])

    # the plain per-pair form: the same pairs, one lsgcpd_register call each
    def per_pair():
        out = []
        for i in range(P):
            out.append(ctx.register(Xd[int(n_off[i]):int(n_off[i + 1])], Yd[int(m_off[i]):int(m_off[i + 1])], p))
        return out
    per_pair()
    flush.zero_()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    singles = per_pair()
    e1.record(stream)
    e1.synchronize()
    pp_ms = e0.elapsed_time(e1)
    pp_pairs = float(sum(s["iters"] * n for s, n in zip(singles, nm)))

    ms, e2e_ms = reduce_max([statistics.mean(step_ms), statistics.mean(e2e_s) * 1e3], ws, "cuda")
    value = job_throughput(pairs_per_step, ws, ms)
    e2e_value = job_throughput(pairs_per_step, ws, e2e_ms)
    t_launch = statistics.mean(estep_ms) / iters_run / 1e3
    per_launch = float(nm.sum())
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = sms * FP32_LANES_PER_SM * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    achieved = FLOPS_PER_PAIR * per_launch / t_launch / 1e12
    roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "traffic": None, "kernel": "estep_kernel (whole batch per launch)",
            "ms_per_launch": round(t_launch * 1e3, 5),
            "launch_timing": "CUDA events around every E-step launch, recorded as nodes of the captured EM graph "
                             "on its stream, in a second timed pass (the headline pass runs without them)", "pairs_per_s_per_launch": per_launch / t_launch,
            "counted": f"{FLOPS_PER_PAIR} FP32-pipe ops + {EX2_PER_PAIR} EX2 per pair, sum N_i M_i pairs per launch",
            "peak_from": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {SM_MAX_MHZ_NOMINAL:.0f} MHz (max SM clock)"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
           "config": {"workload": "batch_256_pairs_500_20000", "pairs": P, "sum_N": int(Ns.sum()),
                      "sum_M": int(Ms.sum()), "sum_NM": int(nm.sum()), "em_iters": iters, "knn_k": 10, "w": 0.1,
                      "alpha_max": 2.0, "lambda": 0.2, "seed": seed,
                      "e_step": "fp32 (packed f32x2) + ex2.approx" if args.precision == 0
                      else "fp32 residuals + f16x2 ex2.approx",
                      "m_step": "double-float Newton (FP32 pairs) on FP64 moments", "l2": "flushed between steps (256 MiB write)",
                      "parallelism": f"replicas x{ws} (independent batches per GPU)"},
           "em_iters_per_s": ws * iters_run / (ms / 1e3),
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": xfer["h2d_bytes"],
                   "d2h_bytes_per_step": xfer["d2h_bytes"], "ms_per_step": round(e2e_ms, 4), "clock": "host wall"},
           "roofline": roof, "clocks": clk, "gpu_launches": launches, "iters_run": iters_run,
           "e_step_plan": plan,
           "per_pair_form": {"value": pp_pairs / (pp_ms / 1e3), "unit": UNIT, "ms_per_step": round(pp_ms, 3),
                             "calls": P, "batched_speedup": round((pp_ms / pp_pairs) / (ms / pairs_per_step), 3)}}
    # the same batch with the moment sums on the tensor cores (precision 2), same protocol
    if args.precision == 0 and not args.no_variants:
        p2 = binding.default_params(max_iters=iters, precision=2)
        for _ in range(max(args.warmup, 1)):
            ctx.register_batch(Xd, n_off, Yd, m_off, p2)
        barrier()
        t2, est2 = [], []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            got2 = ctx.register_batch(Xd, n_off, Yd, m_off, p2)
            e1.record(stream)
            e1.synchronize()
            t2.append(e0.elapsed_time(e1))
        ctx.set_timing(True)  # E-step time per launch from a pass with the per-kernel events
        ctx.register_batch(Xd, n_off, Yd, m_off, p2)
        for _ in range(args.steps):
            flush.zero_()
            ctx.register_batch(Xd, n_off, Yd, m_off, p2)
            torch.cuda.synchronize()
            est2.append(ctx.last_timing()["ms_estep"])
        ctx.set_timing(False)
        barrier()
        ms2 = statistics.mean(t2)
        it2 = int(got2["iters"].max())
        rot = [rotation_angle(got2["R"][i], got["R"][i]) for i in range(P)]
        out["mixed_precision"] = {
            "precision": 2, "e_step": E_STEP_DESC[2], "dtype": DTYPE[2],
            "value": job_throughput(float((got2["iters"].astype(np.float64) * nm).sum()), ws, ms2), "unit": UNIT,
            "ms_per_step": round(ms2, 4), "estep_ms_per_launch": round(statistics.mean(est2) / it2, 5),
            "speedup_vs_fp32_step": round(ms / ms2, 4), "max_rot_err_vs_fp32_rad": float(max(rot))}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the oracle on one pair of the batch (the largest one whose full registration fits the budget)
        order = np.argsort(-nm)
        i = int(order[min(len(order) - 1, 8)])
        q = pairs[i]
        gi = {"R": got["R"][i], "t": got["t"][i], "sigma2": float(got["sigma2"][i])}
        cb, ref = cpu_baseline(q, gi, int(got["iters"][i]), budget_s=30.0)
        cb["sample"] = f"pair {i} of the batch (N={len(q['X'])}, M={len(q['Y'])}): " + cb["sample"]
        out["cpu_baseline"] = cb
        if ref:
            out["vs_fp64_oracle"] = dict(errors_vs(gi, ref, ref["diag"]), pair=i)
    ctx.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    """The FP64 oracle as it stands on this host's cores: each step is one EM
    iteration (E step over a bounded subset of the sources, all targets), sized so
    the whole run stays within a few minutes."""
    import numpy as np

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    name = args.workload if args.workload in SINGLE else "rgbd20k"
    c, seed = workload(0, name)
    X, Y = c["X"], c["Y"]
    N, M = len(X), len(Y)
    pre = oracle.preprocess(Y, 10, 2.0, 0.2)
    V, _ = oracle.volume(Y)
    s2 = oracle.sigma2_init(X, Y, np.eye(3), np.zeros(3))
    # size one step at about 6 s of CPU work
    ns = min(N, 1000)
    t0 = time.perf_counter()
    oracle.estep(X[:ns], Y, pre["normals"], pre["alpha"], np.eye(3), np.zeros(3), s2, 0.1, V)
    rate = ns * M / (time.perf_counter() - t0)
    ns = max(1, min(N, int(6.0 * rate / M)))
    Xs = X[:ns]

    def step():
        o = oracle.estep(Xs, Y, pre["normals"], pre["alpha"], np.eye(3), np.zeros(3), s2, 0.1, V)
        oracle.mstep(o["stats"], Xs, np.eye(3), np.zeros(3))

    for _ in range(max(args.warmup, 0)):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    ms = statistics.mean(times) * 1e3
    value = ns * M / (ms / 1e3)
    cores = os.cpu_count() or 1
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(config_obj(c, seed, args.iters, ws, 0, name), e_step="fp64 (oracle)",
                          m_step="fp64 (oracle)"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"one EM iteration (E step + Newton M step) over {ns} of {N} sources "
                                      f"x {M} targets per step", "cpu": oracle.cpu_model()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch256":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
