"""Benchmark of the HTLR matrix-vector product (HMultVec) on GB300.

Default workload (N=1): d=3, n=32 (N=32768), kernel 1/|x-y|, a(x)=1+0.5 sin(2 pi x_1),
leaf 4^3, Chebyshev order p=5, eta=1, one FP64 right-hand side u ~ N(0,1) (seeded),
STORED layout (one core per admissible block, one dense matrix per inadmissible leaf).
The operator is constructed once (Algorithm 1); a step is one HMultVec (Algorithm 2)
over the whole operator: upward contractions, the stream over every core and dense
block, reductions and the downward expansion into f.

Prints one JSON line.  ``--impl reference`` times the CPU oracle (FP64 C, host cores)
on the same workload instead.
"""
from __future__ import annotations

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

import numpy as np  # noqa: E402

METRIC = "HTLR matvec Gpts*RHS/s"
UNIT = "Gpts*RHS/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="htlr", choices=["htlr", "reference"])
    ap.add_argument("--config", default="c2")
    ap.add_argument("--storage", type=int, default=1, help="1 STORED, 2 SHARED, 0 AUTO")
    ap.add_argument("--far-precision", type=int, default=1, help="0 FP64, 1 DF64, 2 FP32, 3 BF16X6 (tensor cores)")
    ap.add_argument("--near-precision", type=int, default=1, help="0 FP64, 1 DF64, 2 FP32, 3 BF16X6 (tensor cores), 4 TF32X3 (generated, tensor cores)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tc-segment", type=int, default=0,
                    help="tensor-core K steps per accumulator segment (0: library default)")
    ap.add_argument("--tc-flush", type=int, default=0,
                    help="tensor-core segments per FP64 flush (0: library default)")
    ap.add_argument("--gmres-solves", type=int, default=20,
                    help="GMRES solves (to 1e-10) timed after the matvec, per variant")
    ap.add_argument("--cpu-sample-s", type=float, default=20.0)
    ap.add_argument("--paper-tables", action="store_true",
                    help="construct and apply the settings of the paper's Tables 5.1-5.4 "
                         "(context run; prints its own JSON line)")
    ap.add_argument("--paper-max-n-points", type=int, default=1 << 22)
    ap.add_argument("--plan-compare", action="store_true",
                    help="matvec time of htlr_matvec against a captured plan (CUDA graph) on "
                         "c1 and c2")
    ap.add_argument("--solve-large", action="store_true",
                    help="16 second-kind GMRES solves on the c3 grid with a = 1 + 0.5 sin: "
                         "FP64 against df64 residual + BF16X6 inner refinement")
    ap.add_argument("--accuracy", action="store_true",
                    help="c3 and c4 at full size: error of every precision mode against the "
                         "FP64 direct sums on seeded random rows, and the matvec time")
    ap.add_argument("--accuracy-rows", type=int, default=1024)
    ap.add_argument("--accuracy-configs", default="c3,c4")
    ap.add_argument("--accuracy-modes", default="",
                    help="comma list of mode names to run (default: all of the workload's)")
    ap.add_argument("--accuracy-tc-segments", default="",
                    help="comma list of tc_segment values: each BF16X6 mode also runs with "
                         "each of them")
    ap.add_argument("--autotune-ms", type=float, default=2000.0,
                    help="htlr_autotune budget before timing (0: keep the default shapes)")
    ap.add_argument("--serve-requests", type=int, default=32,
                    help="requests of the Poisson serving stream (0: skip serving)")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-max-n2", type=int, default=1024)
    ap.add_argument("--serve-max-n3", type=int, default=128)
    ap.add_argument("--workloads", default="c2_fp64,c3,c4",
                    help="comma list of extra workloads measured after the headline and "
                         "reported under 'workloads' (empty: none)")
    ap.add_argument("--workload-steps", type=int, default=5,
                    help="timed matvecs of each extra workload")
    ap.add_argument("--workload-rows", type=int, default=1024,
                    help="seeded random rows of the FP64 direct sums per extra workload")
    ap.add_argument("--workload-oracle-rows", type=int, default=8,
                    help="rows of the oracle's row-sampled HTLR per extra workload (parity "
                         "and the CPU baseline)")
    return ap.parse_args()


def max_over_ranks(ms, world, device):
    """The slowest rank's step time (ms): every replica's work counts only when all are
    done.  Collective over the default process group when world > 1."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, N, nrhs, ms):
    """Whole-job Gpts*RHS/s of `world` replicas, each applying the operator to N x nrhs
    values per step of `ms` milliseconds (weak scaling: fixed work per GPU)."""
    return world * N * nrhs / (ms * 1e-3) / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dtype_name(info):
    fp, np_ = PREC_NAME[info["far_precision"]], PREC_NAME[info["near_precision"]]
    return fp if fp == np_ else f"{fp} far / {np_} near"


def workload_desc(w, storage_name):
    kern = {0: "log|x-y|", 1: "1/|x-y|", 2: "exp(-|x-y|)", 3: "gauss", 4: "poly", 5: "const"}[w.ktype]
    grid = "uniform grid" if w.grid_kind == "uniform" else "quasi-uniform tensor grid"
    return (f"{w.name}: d={w.d} n={w.n} N={w.N} {grid} kernel {kern} a={w.a_kind} "
            f"leaf {w.leaf}^{w.d} p={w.p} eta={w.eta:.4g} nrhs={w.nrhs} {storage_name}")


def oracle_args(w):
    """Grid arguments of the oracle's HTLR for a workload (tensor grids: no QR)."""
    if w.grid_kind == "uniform":
        return {}
    return {"grid": w.grid(), "orth": False}


# ----------------------------------------------------------------------------------
# clocks sampled with nvidia-smi during the timed region
# ----------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline leg)
# ----------------------------------------------------------------------------------
def time_oracle(w, budget_s):
    """Times the oracle's HMultVec (Algorithm 2, every block's product on all host cores,
    results added in recursion order) on this workload after its construction.  Returns
    (Gpts*RHS/s, cores, sample description, seconds)."""
    import oracle
    cores = oracle.set_num_threads(0)
    t0 = time.perf_counter()
    H = oracle.HTLR(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, a=w.a(), scale=w.kscale, **oracle_args(w),
                    param=w.kparam)
    t_con = time.perf_counter() - t0
    u = w.u(nrhs=1)
    times = []
    t_start = time.perf_counter()
    while True:
        t1 = time.perf_counter()
        f_ref = H.matvec(u)
        times.append(time.perf_counter() - t1)
        if time.perf_counter() - t_start > budget_s or len(times) >= 50:
            break
    H.free()
    time_oracle.last_output = np.asarray(f_ref).reshape(-1)
    t = statistics.median(times)
    val = w.N * 1 / t / 1e9
    sample = (f"oracle construct {t_con:.1f} s, then {len(times)} HMultVec calls on the full "
              f"workload, 1 RHS, {cores} OpenMP threads (host cores), median {t * 1e3:.1f} ms")
    return val, cores, sample, t


def run_reference(args, w):
    """The reference arm: the oracle's HMultVec (Algorithm 2 on every block, all host
    cores) on the same workload; each step is one whole product."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    import oracle as O
    cores = O.set_num_threads(0)
    t0 = time.perf_counter()
    H = O.HTLR(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, a=w.a(), scale=w.kscale, param=w.kparam,
               **oracle_args(w))
    t_con = time.perf_counter() - t0
    u = w.u(nrhs=w.nrhs)
    nrhs = u.shape[1]
    for _ in range(args.warmup):
        H.matvec(u)
    times = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        H.matvec(u)
        times.append(time.perf_counter() - t1)
    H.free()
    t = statistics.mean(times)
    val = w.N * nrhs / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_desc(w, "oracle (per-block)")},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"construct {t_con:.1f} s once; each step one whole "
                                   f"HMultVec (Algorithm 2, every block, {nrhs} RHS) on "
                                   f"{cores} OpenMP threads"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------
PREC_NAME = {0: "f64", 1: "df64", 2: "f32", 3: "bf16x6", 4: "tf32x3"}
PREC_BYTES = {0: 8, 1: 8, 2: 4, 3: 6, 4: 8}
# multiply-adds per second of the stream's inner loop, from unit counts and clocks
# (152 SMs at 2.07 GHz): FP64 2 FMA/clk/SM (the nominal 1.25 TFLOP/s); FP32 128 lanes;
# df64 spends 12 FP32-pipe instructions per multiply-add (see stream_impl.cuh)
ALU_PEAK = {0: 152 * 2 * 2.07e9, 1: 152 * 128 * 2.07e9 / 12, 2: 152 * 128 * 2.07e9}


# DRAM traffic (read + write bytes) of one launch of the dominant kernel, taken with ncu
# on the same workload and kernel build (profiles/stream_kernel_df64_c2_launches.md);
# keyed by (workload, storage, far precision, near precision, RHS).
MEASURED_TRAFFIC = {("c2", 1, 1, 1, 1): 5804274688 + 13374976}


def stream_elements(info, w):
    """Elements (multiply-adds per RHS) of the block stream: every admissible block's core
    (p_eff^d x p_eff^d) and every inadmissible block (|tau| x |sigma|), split into far and
    near, plus the elements actually held (unique blocks, for SHARED storage)."""
    far = far_unique = 0.0
    for lv, nfar in enumerate(info["far_per_level"]):
        if nfar == 0:
            continue
        pe = min(w.p, w.n >> lv)
        far += nfar * float(pe ** w.d) ** 2
    rows = float(w.leaf ** w.d)
    near = info["near_blocks"] * rows * rows
    if info["storage"] == 1:
        far_unique, near_unique = far, near
    else:
        # SHARED: held blocks are the unique ones (bytes_cores / bytes_near already count
        # the padded storage; use them directly)
        far_unique = info["bytes_cores"] / PREC_BYTES[info["far_precision"]]
        near_unique = info["bytes_near"] / PREC_BYTES[info["near_precision"]]
    return far, near, far_unique, near_unique


def stream_roofline(info, w, nrhs, stream_ms, hbm_peak, hbm_src, bf16_peak=None,
                    executed_flops=None):
    fp, np_ = info["far_precision"], info["near_precision"]
    if fp == 3:
        far, near, far_u, near_u = stream_elements(info, w)
        t = stream_ms * 1e-3
        executed = executed_flops          # htlr_tensor_flops: MMAs the matvec issues
        peak = bf16_peak or 1895.3
        useful = 2.0 * (far + (near if np_ == 3 else 0.0)) * nrhs
        held = far_u * PREC_BYTES[fp] + (near_u * PREC_BYTES[np_] if info["storage"] != 3 else 0)
        return {"bound": "tensor", "achieved": executed / t / 1e12, "peak": peak,
                "algorithmic_bytes_per_launch": held, "hbm_achieved_gbs": held / t / 1e9,
                "unit": "TFLOP/s", "frac": executed / t / 1e12 / peak,
                "peak_source": "measured bf16 (MEASURED_PEAKS.json, burst)",
                "kernel": ("tc_group_kernel" if info.get("tc_grouped") else "tc_stream_kernel")
                          + " (tcgen05 kind::f16, BF16x6; stage time includes operand packing)",
                "kernel_ms": stream_ms,
                "executed_tensor_flops_per_launch": executed,
                "useful_fp32_equivalent_tflops": useful / t / 1e12, "traffic": None,
                "precision": {"far": PREC_NAME[fp], "near": PREC_NAME[np_]}}
    far, near, far_u, near_u = stream_elements(info, w)
    t = stream_ms * 1e-3
    hbm_bytes = far_u * PREC_BYTES[fp] + near_u * PREC_BYTES[np_]
    t_hbm = hbm_bytes / (hbm_peak * 1e9)
    t_alu = (far / ALU_PEAK[fp] + near / ALU_PEAK[np_]) * nrhs
    macs = (far + near) * nrhs
    base = {"kernel": "stream_kernel", "kernel_ms": stream_ms,
            "algorithmic_bytes_per_launch": hbm_bytes, "multiply_adds_per_launch": macs,
            "hbm_achieved_gbs": hbm_bytes / t / 1e9,
            "hbm_frac_of_measured": hbm_bytes / t / 1e9 / hbm_peak, "traffic": None,
            "precision": {"far": PREC_NAME[fp], "near": PREC_NAME[np_]}}
    if t_alu > t_hbm:
        peak = 2 * macs / t_alu / 1e12
        ach = 2 * macs / t / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak,
                "peak_source": "derived: 152 SMs x 2.07 GHz x (FP64 2 FMA/clk | FP32 128 "
                               "FMA/clk | df64 128/12 multiply-adds/clk), FP64-equivalent flops"}
    else:
        ach = hbm_bytes / t / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "peak_source": hbm_src}
    roof.update(base)
    return roof


# SFU operations per generated kernel value in FP32 (1/r: rsqrt; exp(-r): rsqrt, ex2;
# Gaussian: ex2; log: lg2), and the SFU rate: 16 per clock per SM, 152 SMs at 2.07 GHz
SFU_PER_PAIR = {0: 1, 1: 1, 2: 2, 3: 1}
SFU_PEAK = 152 * 16 * 2.07e9


def near_tc_roofline(info, w, nrhs, ms):
    """The generated near field on the tensor cores: its bound is the kernel generation on
    the SFUs (the products run on the tensor cores at a few per cent of their rate), so
    achieved = near point pairs (kernel values generated) per second against the SFU rate
    divided by the SFU operations per value."""
    t = ms * 1e-3
    pairs = float(info["near_point_pairs"])
    per = SFU_PER_PAIR.get(w.ktype)
    peak = SFU_PEAK / per / 1e9 if per else None
    ach = pairs / t / 1e9
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Geval/s",
            "frac": ach / peak if peak else None,
            "peak_source": "derived: 152 SMs x 2.07 GHz x 16 SFU ops/clk / %s SFU ops per "
                           "kernel value" % per,
            "kernel": "near_tc_kernel (kernel values generated into tensor memory, "
                      "tcgen05 kind::tf32 products; stage includes packing of w u)",
            "kernel_ms": ms, "multiply_adds_per_launch": pairs * nrhs,
            "tf32_tensor_flops_per_launch": pairs * 16 * ((nrhs + 15) // 16) * 3 * 2,
            "traffic": None, "precision": {"near": PREC_NAME[info["near_precision"]]}}


def near_cc_roofline(info, w, nrhs, ms):
    """The near field on the CUDA cores beside a tensor-core far field, or generated:
    multiply-adds per launch = near point pairs x RHS (plus one kernel evaluation per pair
    when generated), against the pipe of its precision."""
    np_ = info["near_precision"]
    t = ms * 1e-3
    generated = info["storage"] == 3
    pairs = float(info["near_point_pairs"])
    macs = pairs * nrhs
    peak = 2 * ALU_PEAK[np_] / 1e12
    ach = 2 * macs / t / 1e12
    roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "peak_source": "derived: 152 SMs x 2.07 GHz x (FP64 2 | FP32 128 | df64 128/12) "
                           "multiply-adds/clk",
            "kernel": ("near_gen_kernel (kernel values generated per pair)" if generated
                       else "stream_kernel (held near blocks)"), "kernel_ms": ms,
            "multiply_adds_per_launch": macs, "traffic": None,
            "precision": {"near": PREC_NAME[np_]}}
    if generated:
        roof["kernel_evaluations_per_s"] = pairs / t
    return roof


# Extra workloads measured after the headline (name, storage, far and near precision).
SUITE = {
    "c2_fp64": ("c2", 1, 0, 0),     # the headline operator in plain FP64 (STORED)
    "c3": ("c3", 2, 3, 3),          # 64 RHS, SHARED, BF16x6 tensor cores far and near
    "c4": ("c4", 3, 3, 4),          # 16 RHS, tensor grid: BF16x6 far, TF32x3 generated near
}

# DRAM traffic per executed BF16 tensor FLOP of the grouped tensor-core kernel (all its
# launches of one matvec), from ncu on the n = 64 profiling cases of the same operators
# and kernel build (profiles/); the full-size traffic is this ratio times the executed
# FLOPs of the full-size matvec, since every launch streams its cores and sources per
# group and offset.  None: not captured for the current kernel.
TRAFFIC_PER_TENSOR_FLOP = {
    # c3_n64: 18.68 GB of DRAM reads + writes over the three grouped launches of one matvec,
    # 1.482e13 executed BF16 FLOPs (profiles/tc_group_kernel_c3n64_ncu.md)
    "c3": 18.683e9 / 1.4819e13,
    # c4_n64: 19.32 GB over the two grouped launches, 9.680e12 executed FLOPs
    "c4": 19.324e9 / 9.6803e12,
}


def tensor_roofline(info, w, nrhs, stream_ms, bf16_peak, executed_flops):
    """Roofline of the tensor-core stream stage (all grouped launches of one matvec, with
    their operand packing): algorithmic work = the method's multiply-adds (every far core
    p_eff^2d and tensor-core near block |tau||sigma|, per RHS) x 6 split products x 2
    FLOPs, against the measured BF16 peak; the executed fraction (MMA padding included)
    is given beside it."""
    far, near, _, _ = stream_elements(info, w)
    macs = (far + (near if info["near_precision"] == 3 else 0.0)) * nrhs
    t = stream_ms * 1e-3
    alg = 2.0 * 6.0 * macs
    roof = {"bound": "tensor", "achieved": alg / t / 1e12, "peak": bf16_peak, "unit": "TFLOP/s",
            "frac": alg / t / 1e12 / bf16_peak,
            "peak_source": "measured bf16 burst (MEASURED_PEAKS.json)",
            "kernel": "tc_group_kernel (tcgen05 kind::f16, BF16x6; stage includes operand packing)",
            "kernel_ms": stream_ms, "multiply_adds_per_launch": macs,
            "algorithmic_bf16_flops_per_launch": alg,
            "executed_bf16_flops_per_launch": executed_flops,
            "executed_frac": executed_flops / t / 1e12 / bf16_peak, "traffic": None}
    ratio = TRAFFIC_PER_TENSOR_FLOP.get(w.name)
    if ratio:
        roof["traffic"] = ratio * executed_flops
        roof["traffic_source"] = ("ncu dram bytes per executed tensor FLOP on the n=64 case x "
                                  "executed FLOPs here")
    return roof


def run_suite_workload(key, args, stream, peaks, hbm_peak, hbm_src):
    """One extra workload: construct, time `--workload-steps` matvecs (CUDA events on the
    handle's stream), stage times, roofline, error against the FP64 direct sums on seeded
    random rows, parity against the oracle's row-sampled HTLR, and the CPU baseline from
    that oracle's timing."""
    import torch
    import oracle
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    name, storage, fp, np_ = SUITE[key]
    w = workload(name)
    nrhs = w.nrhs
    U = w.u(nrhs=nrhs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, kscale=w.kscale,
                            kparam=w.kparam, a=w.a(), grid=w.grid(), storage=storage,
                            stream=stream, far_precision=fp, near_precision=np_)
    torch.cuda.synchronize()
    construct_s = time.perf_counter() - t0
    out = {}
    try:
        if name == "c2":
            htlr.htlr_autotune(H, nrhs=nrhs, budget_ms=1000.0)
        info = htlr.htlr_info(H)
        storage_name = ({1: "STORED", 2: "SHARED", 3: "GENERATED"}[info["storage"]] + " " +
                        dtype_name(info))
        with torch.cuda.stream(stream):
            ud = torch.from_numpy(np.ascontiguousarray(U.T)).cuda()
            fd = torch.empty_like(ud)
            flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        for _ in range(2):
            htlr.htlr_matvec(H, ud, fd, nrhs)
        htlr.htlr_sync(H)
        steps = args.workload_steps if name != "c2" else max(args.workload_steps, 20)
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        time.sleep(0.3)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.fill_(float(k))             # evicts L2 (256 MB > 129 MB)
                ev[k][0].record(stream)
                htlr.htlr_matvec(H, ud, fd, nrhs)
                ev[k][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        htlr.htlr_sync(H)                         # a device check that failed voids the line
        launches = htlr.htlr_last_launch_count(H) * steps
        ms = [a.elapsed_time(b) for a, b in ev]
        mean_ms = float(np.mean(ms))
        stage = np.zeros(5)
        nst = 3 if name != "c2" else 10
        for k in range(nst):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
            stage += np.array(htlr.htlr_matvec_timed(H, ud, fd, nrhs))
        stage_ms = stage / nst
        roofs = []
        if fp == 3:
            roofs.append(tensor_roofline(info, w, nrhs, stage_ms[1], peaks.get("bf16_tflops", 1885.6),
                                         htlr.htlr_tensor_flops(H, nrhs)))
        else:
            roofs.append(stream_roofline(info, w, nrhs, stage_ms[1], hbm_peak, hbm_src))
        if stage_ms[2] > 1e-2:
            roofs.append(near_tc_roofline(info, w, nrhs, stage_ms[2]) if np_ == 4 else
                         near_cc_roofline(info, w, nrhs, stage_ms[2]))
        roofs.sort(key=lambda r: -r["kernel_ms"])
        # the timed product's rows (the last timed matvec left f in fd)
        rows = w.sample_rows(args.workload_rows, seed=1024) if w.N > 100000 else None
        with torch.cuda.stream(stream):
            f_all = fd.cpu().numpy().T
        torch.cuda.synchronize()
        out = {
            "workload": workload_desc(w, storage_name), "nrhs": nrhs,
            "value": w.N * nrhs / (mean_ms * 1e-3) / 1e9, "unit": UNIT,
            "matvec_ms": {"mean": mean_ms, "median": float(np.median(ms)), "min": float(min(ms)),
                          "steps": steps},
            "l2": ("flushed between steps (256 MB write)" if w.N * nrhs * 8 < 129e6 else
                   "u and f (%.2f GB each) exceed L2; flushed between steps as well" %
                   (w.N * nrhs * 8 / 1e9)),
            "construct_s": construct_s,
            "stage_ms": {"up": stage_ms[0], "stream": stage_ms[1], "near_cuda_cores": stage_ms[2],
                         "reduce": stage_ms[3], "out": stage_ms[4]},
            "roofline": roofs[0], "roofline_other": roofs[1:], "clocks": clk,
            "gpu_launches": launches, "bytes_held": info["bytes_total"],
        }
    finally:
        htlr.htlr_free(H)
    # ---- CPU side: parity and accuracy on sampled rows, and the oracle's timing ----
    cores = oracle.set_num_threads(0)
    okw = oracle_args(w)
    if rows is None:
        # small operator: the whole oracle HTLR (every row) and its HMultVec time
        val, cores, sample, t = time_oracle(w, min(args.cpu_sample_s, 5.0))
        ref = time_oracle.last_output
        out["parity_vs_oracle_htlr"] = {"rel_err": float(np.linalg.norm(f_all[:, 0] - ref) /
                                                         np.linalg.norm(ref)),
                                        "tolerance": 1e-12, "compared": "RHS 1, all N rows"}
        out["cpu_baseline"] = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": sample}
        return out
    t0 = time.perf_counter()
    ref = oracle.dense_rows(w.d, w.n, w.ktype, U, rows, scale=w.kscale, param=w.kparam,
                            grid=w.grid(), a=w.a(), q=w.q)
    t_dense = time.perf_counter() - t0
    out["error_vs_direct_sums"] = dict(_col_rel(f_all[rows], ref), rows=int(len(rows)),
                                       rhs=nrhs, direct_sums_s=t_dense, cores=cores)
    orows = w.sample_rows(args.workload_oracle_rows, seed=4096)
    t0 = time.perf_counter()
    oref = oracle.htlr_rows(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, U, orows, scale=w.kscale,
                            param=w.kparam, a=w.a(), **okw)
    t_rows = time.perf_counter() - t0
    out["parity_vs_oracle_htlr"] = dict(_col_rel(f_all[orows], oref), rows=int(len(orows)),
                                        rhs=nrhs)
    out["cpu_baseline"] = {"value": len(orows) * nrhs / t_rows / 1e9, "unit": UNIT,
                           "cores": cores, "kind": "oracle",
                           "sample": f"row-sampled oracle HTLR (Algorithms 1-2 on every block "
                                     f"of the sampled rows' target boxes): {len(orows)} rows x "
                                     f"{nrhs} RHS in {t_rows:.1f} s on {cores} OpenMP threads; "
                                     f"rows x RHS per second, extrapolated per row"}
    return out


def time_gmres(w, solves, stream):
    """Solve latency of a(x)u + Ku = f to 1e-10 (GMRES(30) from u = 0, seeded f ~ N(0,1)):
    plain FP64 operator versus df64 residual operator with an FP32 far field inner
    operator (iterative refinement).  Each solve is timed with CUDA events."""
    import torch
    from paper_2508_05958_gb300 import htlr
    out = {}
    # operators held SHARED (one block per offset): the faster single-RHS form for every
    # precision here, the plain FP64 baseline included
    variants = {"fp64": ((0, 0), None), "mixed_refined": ((1, 1), (2, 1))}
    for name, (acc, inner) in variants.items():
        H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, kscale=w.kscale,
                                kparam=w.kparam, a=w.a(), far_precision=acc[0],
                                near_precision=acc[1], stream=stream, storage=2)
        Hi = None
        if inner:
            Hi = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, kscale=w.kscale,
                                     kparam=w.kparam, a=w.a(), far_precision=inner[0],
                                     near_precision=inner[1], stream=stream, storage=2)
        f = torch.from_numpy(np.ascontiguousarray(w.u(nrhs=1, seed=500).T)).cuda()
        u = torch.zeros_like(f)
        htlr.htlr_gmres(H, f, u, 1, H_inner=Hi)          # warm-up
        times, res = [], None
        for k in range(solves):
            f = torch.from_numpy(np.ascontiguousarray(w.u(nrhs=1, seed=501 + k).T)).cuda()
            u.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = htlr.htlr_gmres(H, f, u, 1, H_inner=Hi)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        htlr.htlr_free(H)
        if Hi:
            htlr.htlr_free(Hi)
        times.sort()
        out[name] = {"p50_ms": times[len(times) // 2],
                     "p99_ms": times[min(len(times) - 1, int(0.99 * len(times)))],
                     "solves_per_s": 1e3 / float(np.mean(times)), "iterations": res["iterations"],
                     "refinements": res["refinements"], "rel_residual": res["rel_residual"]}
    return out


def time_serving(args):
    """Continuous-batching solve server against FP64 one-at-a-time on the same seeded
    Poisson stream of GMRES(30) solves to 1e-10 (operators warmed: one solve each first)."""
    from paper_2508_05958_gb300 import htlr, serving
    ops = serving.family(max_n2=args.serve_max_n2, max_n3=args.serve_max_n3)
    stream = serving.request_stream(ops, args.serve_rate, args.serve_requests, seed=2025)
    arms = {"fp64_one_at_a_time": dict(mixed=0, max_active=1, max_batch=1),
            "mixed_batched": dict(mixed=1, inner_precision=htlr.PREC_FP32, max_active=64,
                                  max_batch=16),
            "mixed_batched_tensor_cores": dict(mixed=1, inner_precision=htlr.PREC_BF16X6,
                                               inner_tol=1e-5, max_active=64, max_batch=16)}
    out = {"workload": f"{len(ops)} operators (d=2 n<={args.serve_max_n2} log; d=3 "
                       f"n<={args.serve_max_n3} 1/r, exp(-r); r in 5..7; SHARED), "
                       f"{args.serve_requests} requests, Poisson {args.serve_rate:g}/s, "
                       "f ~ N(0,1), GMRES(30) to 1e-10",
           "latency": "p50/p99: submission to completion (includes queueing behind earlier "
                      "requests); service_*: admission to completion; queue_*: submission to "
                      "admission"}
    for name, kw in arms.items():
        with htlr.Server(**kw) as S:
            ids = [S.add_operator(o.ktype, o.d, o.n, o.leaf, o.r, o.eta, a=o.a(), storage=2)
                   for o in ops]
            # warm: construct every operator (a zero right-hand side finishes after the
            # first residual, one matvec)
            for k, o in enumerate(ops):
                S.wait(S.submit(ids[k], np.zeros(o.N)))
            res = serving.replay(S, ops, stream, op_ids=ids)
            st = S.stats()
        res["batched_matvecs"] = st["batched_matvecs"]
        res["mean_columns_per_matvec"] = st["matvec_columns"] / max(1, st["batched_matvecs"])
        res["max_batch_seen"] = st["max_batch_seen"]
        out[name] = res
    out["solves_per_s_ratio"] = (out["mixed_batched"]["solves_per_s"] /
                                 out["fp64_one_at_a_time"]["solves_per_s"])
    out["solves_per_s_ratio_tensor_cores"] = (out["mixed_batched_tensor_cores"]["solves_per_s"] /
                                              out["fp64_one_at_a_time"]["solves_per_s"])
    return out


def run_gpu(args, w):
    import torch
    from paper_2508_05958_gb300 import htlr
    rank, world, local = dist_env()
    dev = local if torch.cuda.device_count() > local else 0
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    stream = torch.cuda.Stream()
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"

    t0 = time.perf_counter()
    H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, kscale=w.kscale,
                            kparam=w.kparam, a=w.a(), grid=w.grid(), storage=args.storage,
                            stream=stream, tc_segment=args.tc_segment, tc_flush=args.tc_flush,
                            far_precision=args.far_precision, near_precision=args.near_precision)
    torch.cuda.synchronize()
    construct_s = time.perf_counter() - t0
    tune = None
    if args.autotune_ms > 0:
        tune = htlr.htlr_autotune(H, nrhs=w.nrhs, budget_ms=args.autotune_ms)
    info = htlr.htlr_info(H)
    storage_name = ({1: "STORED", 2: "SHARED", 3: "GENERATED"}.get(info["storage"], "?") + " " +
                    dtype_name(info))
    nrhs = w.nrhs
    U = w.u(nrhs=nrhs)
    with torch.cuda.stream(stream):
        ud = torch.from_numpy(np.ascontiguousarray(U.T)).cuda()
        fd = torch.empty_like(ud)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    for _ in range(max(3, args.warmup)):
        htlr.htlr_matvec(H, ud, fd, nrhs)
    torch.cuda.synchronize()
    launches_per_step = htlr.htlr_last_launch_count(H)

    # timed region: per-step CUDA events on the handle's stream, L2 flushed between steps
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))                 # evicts L2 (256 MB > 129 MB)
            ev[k][0].record(stream)
            htlr.htlr_matvec(H, ud, fd, nrhs)     # asynchronous, on the same stream
            ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    # a device check that failed inside the timed region (a bounded wait that ran out)
    # voids the measurement: htlr_sync raises and no line is printed
    htlr.htlr_sync(H)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(float(np.mean(step_ms)), world, "cuda")
    value = replica_throughput(world, w.N, nrhs, ms)
    # stage breakdown (events around each stage), from separate L2-flushed passes
    stage, nst = np.zeros(5), max(3, min(args.steps, 20))
    for k in range(nst):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        stage += np.array(htlr.htlr_matvec_timed(H, ud, fd, nrhs))
    stage_ms = stage / nst

    # roofline of the dominant kernel (the block stream)
    roofs = [stream_roofline(info, w, nrhs, stage_ms[1], hbm_peak, hbm_src,
                             peaks.get("bf16_tflops"), htlr.htlr_tensor_flops(H, nrhs))]
    if stage_ms[2] > 1e-2:            # near field (CUDA or tensor cores) in its own stage
        roofs.append(near_tc_roofline(info, w, nrhs, stage_ms[2]) if info["near_precision"] == 4
                     else near_cc_roofline(info, w, nrhs, stage_ms[2]))
    roofs.sort(key=lambda r: -r["kernel_ms"])
    roof = roofs[0]                   # the dominant kernel
    key = (w.name, info["storage"], info["far_precision"], info["near_precision"], nrhs)
    if key in MEASURED_TRAFFIC and roof["kernel"] == "stream_kernel":
        roof["traffic"] = MEASURED_TRAFFIC[key]
        roof["traffic_source"] = "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch"

    # end to end through the host-buffer entry point (pinned host memory, copies timed)
    uh = torch.from_numpy(np.ascontiguousarray(U.T)).pin_memory().numpy()
    fh = torch.empty(uh.shape, dtype=torch.float64).pin_memory().numpy()
    for _ in range(2):
        htlr.htlr_matvec_host(H, uh, fh, nrhs)
    e2e_times = []
    for _ in range(max(3, min(args.steps, 20))):
        t1 = time.perf_counter()
        htlr.htlr_matvec_host(H, uh, fh, nrhs)
        e2e_times.append(time.perf_counter() - t1)
    e2e_s = float(np.mean(e2e_times))
    io_bytes = w.N * nrhs * 8

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype_name(info), "data": "synthetic",
        "config": {"workload": workload_desc(w, storage_name), "l2": "flushed between steps "
                   "(256 MB write); block bytes held: %.3f GB" % (
                       (info["bytes_cores"] + info["bytes_near"]) / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "construct_s": construct_s, "autotune": tune, "stage_ms": {"up": stage_ms[0],
                   "stream": stage_ms[1], "near_cuda_cores": stage_ms[2],
                   "reduce": stage_ms[3], "out": stage_ms[4]},
                   "bytes_total": info["bytes_total"], "far_per_level": info["far_per_level"],
                   "near_blocks": info["near_blocks"]},
        "roofline": roof,
        "roofline_other": roofs[1:],
        "e2e": {"value": w.N * nrhs / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": io_bytes,
                "d2h_bytes_per_step": io_bytes, "entry_point": "htlr_matvec_host"},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
    }
    f_head = fd[0].double().cpu().numpy()             # first RHS of the last timed matvec
    if world == 1 and args.workloads:
        line["workloads"] = {k: run_suite_workload(k, args, stream, peaks, hbm_peak, hbm_src)
                             for k in args.workloads.split(",") if k}
    if args.gmres_solves > 0 and w.a_kind != "zero":
        line["gmres"] = time_gmres(w, args.gmres_solves, stream)
    if args.serve_requests > 0 and world == 1:
        line["serving"] = time_serving(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        f_gpu = f_head
        val, cores, sample, _ = time_oracle(w, args.cpu_sample_s)
        f_ref = time_oracle.last_output
        tol = {0: 1e-12, 1: 1e-12, 2: 1e-6, 3: 1e-6, 4: 1e-6}[max(info["far_precision"],
                                                        info["near_precision"])]
        line["cpu_baseline"] = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": sample,
                                "parity": {"rel_err_vs_oracle_htlr": float(
                                    np.linalg.norm(f_gpu - f_ref) / np.linalg.norm(f_ref)),
                                    "tolerance": tol, "compared": "RHS 1, all N rows"}}
    htlr.htlr_free(H)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# Settings of the paper's Tables 5.1-5.4 (§5.2, §5.3): table, kernel, d, n, leaf, p,
# admissibility, storage m_h (GB) and MATLAB construction time t_c (s) as printed there
# (one Xeon Gold 6226R).  Gaussian sigma = sqrt(d); SLP = -log r / (2 pi) in 2D and
# 1 / (4 pi r) in 3D; strong admissibility = non-adjacent (eta = sqrt(d)); a = 0.
PAPER_ROWS = [
    ("5.1", "gauss", 2, 256, 16, 8, "weak", 0.16, 1.5), ("5.1", "gauss", 2, 512, 16, 8, "weak", 0.65, 3.8),
    ("5.1", "gauss", 2, 1024, 16, 8, "weak", 2.6, 16), ("5.1", "gauss", 2, 2048, 16, 8, "weak", 10, 68),
    ("5.1", "gauss", 2, 4096, 16, 8, "weak", 41, 280), ("5.1", "gauss", 2, 8192, 16, 8, "weak", 170, 1100),
    ("5.2", "slp", 2, 256, 16, 8, "strong", 1.3, 7.6), ("5.2", "slp", 2, 512, 16, 8, "strong", 5.4, 30),
    ("5.2", "slp", 2, 1024, 16, 8, "strong", 23, 130), ("5.2", "slp", 2, 2048, 16, 8, "strong", 92, 540),
    ("5.2", "slp", 2, 4096, 16, 8, "strong", 370, 2100),
    ("5.3", "gauss", 3, 32, 4, 4, "weak", 0.14, 4.0), ("5.3", "gauss", 3, 64, 4, 4, "weak", 1.2, 27),
    ("5.3", "gauss", 3, 128, 4, 4, "weak", 9.2, 220), ("5.3", "gauss", 3, 256, 4, 4, "weak", 74, 1800),
    ("5.3", "gauss", 3, 512, 4, 4, "weak", 590, 15000),
    ("5.4", "slp", 3, 32, 4, 4, "strong", 2.1, 48), ("5.4", "slp", 3, 64, 4, 4, "strong", 23, 540),
    ("5.4", "slp", 3, 128, 4, 4, "strong", 210, 5100),
]


def run_paper_tables(args):
    """Construct (SHARED, FP64) and apply (one RHS) each setting of the paper's tables up to
    --paper-max-n-points points; report GPU construction and matvec times beside the
    paper's construction times, and the storage of the paper's layout (m_h) beside the
    printed m_h.  Context only: the paper's code is MATLAB on one CPU socket."""
    import torch
    from paper_2508_05958_gb300 import htlr
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    rows = []
    for (tab, kern, d, n, leaf, p, adm, mh, tc) in PAPER_ROWS:
        N = n ** d
        if N > args.paper_max_n_points:
            continue
        if kern == "gauss":
            ktype, scale, param = 3, 1.0, math.sqrt(d)
        else:
            ktype, scale, param = (0, -1.0 / (2 * math.pi), 0.0) if d == 2 else (1, 1.0 / (4 * math.pi), 0.0)
        eta = 0.0 if adm == "weak" else math.sqrt(d)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = htlr.htlr_construct(ktype, d, n, leaf, p, eta, kscale=scale, kparam=param,
                                storage=2, stream=stream)
        torch.cuda.synchronize()
        t_con = time.perf_counter() - t0
        info = htlr.htlr_info(H)
        with torch.cuda.stream(stream):
            u = torch.randn(1, N, dtype=torch.float64, device="cuda")
            f = torch.empty_like(u)
            for _ in range(3):
                htlr.htlr_matvec(H, u, f, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                htlr.htlr_matvec(H, u, f, 1)
            e1.record(stream)
        torch.cuda.synchronize()
        mv_ms = e0.elapsed_time(e1) / 5
        htlr.htlr_free(H)
        rows.append({"table": tab, "kernel": kern, "d": d, "N": N, "p": p, "admissibility": adm,
                     "gpu_construct_s": t_con, "paper_tc_s": tc,
                     "m_h_GiB": info["paper_storage_doubles"] * 8 / 2 ** 30, "paper_m_h_GB": mh,
                     "held_GB": info["bytes_total"] / 1e9, "gpu_matvec_fp64_ms": mv_ms,
                     "Gpts_per_s": N / (mv_ms * 1e-3) / 1e9})
    print(json.dumps({"paper_tables": rows, "note": "paper times: MATLAB R2023b, one Xeon "
                      "Gold 6226R (construction only; its matvec times are plots); GPU: "
                      "SHARED storage, FP64, one RHS, CUDA events"}), flush=True)


def run_solve_large(args):
    """One batch of 16 GMRES(30) solves of a u + K u = f to 1e-10 on the c3 grid
    (N = 2,097,152, 1/|x-y|, a = 1 + 0.5 sin 2 pi x_1): SHARED FP64 operator against the
    df64 residual operator with a BF16X6 tensor-core inner operator (refinement)."""
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    torch.cuda.set_device(0)
    w = workload("c3", a_kind="sin", nrhs=16)
    stream = torch.cuda.Stream()
    f = torch.from_numpy(np.ascontiguousarray(w.u(nrhs=16).T)).cuda()
    out = {"workload": workload_desc(w, "SHARED"), "rhs": 16}
    for name, acc, inner in (("mixed_refined_tensor_cores", (1, 1), (3, 3)), ("fp64", (0, 0), None)):
        H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, a=w.a(), storage=2,
                                far_precision=acc[0], near_precision=acc[1], stream=stream)
        Hi = None
        if inner:
            Hi = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, a=w.a(), storage=2,
                                     far_precision=inner[0], near_precision=inner[1],
                                     stream=stream)
        u = torch.zeros_like(f)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = htlr.htlr_gmres(H, f, u, 16, H_inner=Hi, inner_tol=1e-5)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"seconds": dt, "solves_per_s": 16 / dt, **res}
        htlr.htlr_free(H)
        if Hi:
            htlr.htlr_free(Hi)
    out["speedup"] = out["fp64"]["seconds"] / out["mixed_refined_tensor_cores"]["seconds"]
    print(json.dumps({"solve_large": out}), flush=True)


# precision modes (name, storage, far precision, near precision) of the accuracy run: the
# plain FP64 path first, then the mixed ones; c4's tensor grid takes the generated near field
ACCURACY_MODES = {
    "c3": [("fp64", 2, 0, 0), ("df64", 2, 1, 1), ("f32 far / df64 near", 2, 2, 1),
           ("bf16x6 far / df64 near", 2, 3, 1), ("bf16x6", 2, 3, 3)],
    "c4": [("fp64", 3, 0, 0), ("bf16x6 far / f64 near", 3, 3, 0), ("f32", 3, 2, 2),
           ("bf16x6 far / f32 near", 3, 3, 2), ("bf16x6 far / tf32x3 near", 3, 3, 4)],
}


def _col_rel(f, ref):
    """Per-column relative 2-norm errors over the sampled rows: (max, median)."""
    e = np.linalg.norm(f - ref, axis=0) / np.linalg.norm(ref, axis=0)
    return {"max": float(e.max()), "median": float(np.median(e))}


def run_accuracy(args):
    """Full-size error of every precision mode against the FP64 direct sums (the dense
    Nystrom product, eq. (1.3)-(1.4)) on seeded random rows: c3 with its 64 RHS, c4 with
    its 16.  The direct sums come from the CPU oracle (OpenMP, all host cores) before the
    GPU is touched; each mode's matvec is timed with CUDA events (a single run for the
    slow modes, the median of three after a warm-up for the fast ones)."""
    import oracle
    out = []
    for name in [c for c in args.accuracy_configs.split(",") if c]:
        from paper_2508_05958_gb300.workloads import workload
        w = workload(name)
        u = w.u(nrhs=w.nrhs)
        rows = w.sample_rows(args.accuracy_rows, seed=1024)
        t0 = time.perf_counter()
        ref = oracle.dense_rows(w.d, w.n, w.ktype, u, rows, scale=w.kscale, param=w.kparam,
                                grid=w.grid(), a=w.a(), q=w.q)
        t_dense = time.perf_counter() - t0
        out.append({"w": w, "u": u, "rows": rows, "ref": ref, "t_dense": t_dense})
    import torch
    from paper_2508_05958_gb300 import htlr
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    res_all = []
    for item in out:
        w, u, rows, ref = item["w"], item["u"], item["rows"], item["ref"]
        ud = torch.from_numpy(np.ascontiguousarray(u.T)).cuda()
        fd = torch.empty_like(ud)
        rows_d = torch.from_numpy(rows).cuda()
        res = {"workload": workload_desc(w, "").strip(), "rows": int(len(rows)),
               "rhs": int(u.shape[1]), "direct_sums_s": item["t_dense"],
               "direct_sums_cores": oracle.num_threads(), "modes": []}
        f64 = None
        modes = [(m, st, fp, np_, 0) for m, st, fp, np_ in ACCURACY_MODES.get(w.name, [])]
        if args.accuracy_modes:
            keep = set(args.accuracy_modes.split(","))
            modes = [m for m in modes if m[0] in keep]
        segs = [int(v) for v in args.accuracy_tc_segments.split(",") if v]
        modes += [(f"{m} (tc_segment {sg})", st, fp, np_, sg) for m, st, fp, np_, _ in modes
                  if fp == 3 for sg in segs]
        for mname, storage, fp, np_, seg in modes:
            H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, kscale=w.kscale,
                                    kparam=w.kparam, a=w.a(), grid=w.grid(), storage=storage,
                                    stream=stream, far_precision=fp, near_precision=np_,
                                    tc_segment=seg)
            try:
                info = htlr.htlr_info(H)
                times = []
                for k in range(4):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    htlr.htlr_matvec(H, ud, fd, u.shape[1])
                    e1.record(stream)
                    htlr.htlr_sync(H)
                    times.append(e0.elapsed_time(e1))
                    if times[0] > 2000.0:
                        break
                ms = times[0] if len(times) == 1 else statistics.median(times[1:])
                with torch.cuda.stream(stream):
                    fr = fd.index_select(1, rows_d).cpu().numpy().T.copy()
            finally:
                htlr.htlr_free(H)
            m = {"mode": mname, "storage": {1: "STORED", 2: "SHARED", 3: "GENERATED"}[info["storage"]],
                 "matvec_ms": ms, "rel_err_vs_direct_sums": _col_rel(fr, ref)}
            if mname == "fp64":
                f64 = fr
            elif f64 is not None:
                m["rel_diff_vs_gpu_fp64"] = _col_rel(fr, f64)
            res["modes"].append(m)
            print(json.dumps({"accuracy_mode": w.name, **m}), flush=True)
        res_all.append(res)
    print(json.dumps({"accuracy": res_all}), flush=True)


def run_plan_compare(args):
    """Back-to-back matvecs (warm L2, CUDA events around 200 of them) issued one call at a
    time with htlr_matvec, and replayed from a plan (one CUDA graph launch each)."""
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    torch.cuda.set_device(0)
    out = []
    for name, storage, prec in (("c1", 1, 0), ("c2", 2, 1), ("c2", 1, 1)):
        w = workload(name)
        stream = torch.cuda.Stream()
        H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, a=w.a(), storage=storage,
                                far_precision=prec, near_precision=prec, stream=stream)
        u = torch.from_numpy(np.ascontiguousarray(w.u(nrhs=1).T)).cuda()
        f = torch.empty_like(u)
        P = htlr.htlr_plan_create(H, u, f, 1)
        res = {"workload": workload_desc(w, {1: "STORED", 2: "SHARED"}[storage] + " " +
                                         PREC_NAME[prec]),
               "launches_per_matvec": htlr.htlr_plan_launches(P)}
        for mode in ("htlr_matvec", "plan"):
            run = (lambda: htlr.htlr_matvec(H, u, f, 1)) if mode == "htlr_matvec" else \
                  (lambda: htlr.htlr_plan_launch(P))
            with torch.cuda.stream(stream):
                for _ in range(20):
                    run()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(200):
                    run()
                e1.record(stream)
            torch.cuda.synchronize()
            res[mode + "_us"] = e0.elapsed_time(e1) / 200 * 1e3
        htlr.htlr_plan_free(P)
        htlr.htlr_free(H)
        out.append(res)
    print(json.dumps({"plan_compare": out}), flush=True)


def main():
    args = parse()
    if args.accuracy:
        run_accuracy(args)
        return
    if args.plan_compare:
        run_plan_compare(args)
        return
    if args.solve_large:
        run_solve_large(args)
        return
    if args.paper_tables:
        run_paper_tables(args)
        return
    from paper_2508_05958_gb300.workloads import workload
    w = workload(args.config)
    if args.impl == "reference":
        run_reference(args, w)
        return
    run_gpu(args, w)


if __name__ == "__main__":
    main()
