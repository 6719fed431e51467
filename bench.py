#!/usr/bin/env python3
"""Benchmark of the CRS spMVM C = A*B on GB300.

Default workload: the 3D 7-point variable-coefficient Poisson stencil on a
280^3 grid (N = 21,952,000 rows, 153,193,600 nonzeros, FP64 CRS), the stand-in
for the paper's sAMG matrix.  One step = one product C = A*B with the plan's
default kernel (CRS_L1: thread per row; the val/col slices of the CTA 456
positions ahead are prefetched into L2 by the TMA engine).  Inputs (2.28 GB)
exceed L2 (129 MB), so no flush is needed between steps.

--workload powerlaw_batch512: 512 uneven power-law matrices with k = 4
right-hand sides each, one step = one batched persistent launch (graph
replay) with the adaptive row policy and the autotuned configuration.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle instead.
Under torchrun each rank runs an independent replica (the product does not
shard over GPUs here) and `value` is the sum over ranks.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spMVM GFlop/s & HBM GB/s vs roofline; chosen form vs plain CRS at stated err"
WORKLOADS = {
    "poisson3d_280": "3D 7-point variable-coefficient Poisson stencil, 280^3 grid, N=21,952,000, nnz=153,193,600, "
                     "FP64 CRS, B~U[-1,1) seed 0",
    "poisson3d_160": "3D 7-point variable-coefficient Poisson stencil, 160^3 grid, N=4,096,000, nnz=28,518,400, "
                     "FP64 CRS (profiling size)",
    "eigen_6201600": "symmetric eigenproblem-shaped matrix, N=6,201,600 (400 x 15,504), ~13.8 nnz/row, FP64 CRS",
    "laplace2d_256": "2D 5-point Laplacian 256^2, N=65,536, nnz=326,656, FP64 CRS (L2 resident)",
    "powerlaw_batch512": "512 matrices, N log-uniform in [1e3,2e5], power-law rows (alpha 2.2, 1..2000), "
                         "uniform columns, k=4 RHS each, one persistent graph-captured launch",
}
VARIANTS = {"crs_staged": (1, 1), "crs_l1": (2, 1), "crs_l2": (3, 1), "crs_l4": (4, 1), "crs_l8": (5, 1),
            "crs_l16": (6, 1), "crs_l32": (7, 1), "sell_s1": (8, 1), "sell_s256": (8, 256), "sell_s4096": (8, 4096),
            "sym": (9, 1)}
# FP64 rate from unit counts and the highest SM clock: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz.
# Context only: the roofs below use the rate the FP64 probe measures on the device in the same run.
FP64_UNIT_COUNT_GFLOPS = 152 * 2 * 2 * 2.07
MACHINE = {"fp64_gflops": FP64_UNIT_COUNT_GFLOPS, "fp64_kind": "unit count (probe not run)"}


def fp64_peak() -> float:
    """FP64 FMA rate (GFLOP/s) used as the ALU roof: the probe's measurement."""
    return MACHINE["fp64_gflops"]


# The paper's own single-socket CRS numbers (Sec. 2), quoted as context only: other hardware,
# other (real) matrix; its multi-node results (QDR-InfiniBand Westmere cluster, Cray XE6) exist
# only as figures.
PAPER_CONTEXT = {"hardware": "Intel Xeon X5550 (Nehalem EP), one socket, 4 cores, 3 x DDR3-1333",
                 "matrix": "HMeP Hamiltonian, N = 6.2e6, Nnzr ~ 15, FP64 CRS",
                 "spmvm_gflops": 2.25, "spmvm_gbs": 18.1, "model_limit_gflops_at_spmvm_bw": 2.66,
                 "kappa_bytes_per_nnz": 2.5, "hmep_kappa": 3.79,
                 "multi_node": "QDR-InfiniBand Westmere cluster and Cray XE6: figures only, no numbers",
                 "note": "context, not a target: no vs_baseline is computed from it"}


def sm_max_mhz() -> float:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            v = json.load(f).get("sm_max_mhz")
            if v:
                return float(v)
    return 2070.0


def probe_machine(spmv) -> dict:
    """Secondary roofs measured by the library's own probe kernels in this run.
    Each probe also reads the SM clock it ran at (clock cycles over globaltimer
    nanoseconds), so its rate per SM and clock is known; the roofs are that
    rate at the highest SM clock (the clock the bench's kernels run at):
      FP64: FMAs per SM and clock (spmv_probe_fp64);
      requests: random 8-byte reads per SM and clock out of an L2-resident
                buffer the size of the eigenproblem matrix's B
                (spmv_probe_gather); each is one request from the SM's L1 to
                the crossbar, the port that bounds scattered gathers.
    The HBM copy peak is the measured one of MEASURED_PEAKS.json."""
    f = spmv.spmv_probe_fp64(5)
    l2 = spmv.spmv_probe_gather(6_201_600, 5)
    dram = spmv.spmv_probe_gather(1 << 28, 3)
    hbm, kind = measured_hbm()
    sms, fmax = f["sm_count"], sm_max_mhz()
    fma_clk = f["gflops"] * 1e3 / (2 * sms * f["sm_mhz"])
    req_clk = l2["gathers_per_s"] / (sms * l2["sm_mhz"] * 1e6)
    MACHINE.update({"fp64_gflops": fma_clk * 2 * sms * fmax / 1e3,
                    "fp64_kind": f"measured: {fma_clk:.3f} FMA per SM and clock (spmv_probe_fp64) x {sms} SMs "
                                 f"x 2 flop x {fmax:.0f} MHz",
                    "l2_gathers_per_s": req_clk * sms * fmax * 1e6,
                    "dram_gathers_per_s": dram["gathers_per_s"]})
    return {"sm_count": sms, "sm_max_mhz": fmax,
            "fp64": {"probe_gflops": round(f["gflops"], 1), "probe_sm_mhz": round(f["sm_mhz"], 1),
                     "fma_per_sm_per_clock": round(fma_clk, 4),
                     "peak_gflops_at_max_clock": round(MACHINE["fp64_gflops"], 1),
                     "unit_count_gflops": round(FP64_UNIT_COUNT_GFLOPS, 1)},
            "random_reads_l2": {"probe_per_s": round(l2["gathers_per_s"] / 1e9, 2), "unit": "1e9 per s",
                                "probe_sm_mhz": round(l2["sm_mhz"], 1),
                                "per_sm_per_clock": round(req_clk, 4),
                                "peak_at_max_clock": round(MACHINE["l2_gathers_per_s"] / 1e9, 2)},
            "random_reads_hbm": {"probe_per_s": round(dram["gathers_per_s"] / 1e9, 2), "unit": "1e9 per s",
                                 "buffer_bytes": 8 << 28},
            "hbm_gbs": hbm, "hbm_kind": kind,
            "how": "spmv_probe_fp64: 8 FMA chains per thread with register operands, all SMs; "
                   "spmv_probe_gather: random 8-byte read-only loads, 8 in flight per thread, over 6,201,600 "
                   "doubles (50 MB, L2-resident) and 2^28 doubles (2 GB); best of 5 / 3 launches"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="poisson3d_280", choices=sorted(WORKLOADS))
    ap.add_argument("--variant", default="crs_l1", choices=sorted(VARIANTS))
    ap.add_argument("--fp32-val", action="store_true", help="store val in FP32 (FP64 accumulation)")
    ap.add_argument("--k", type=int, default=1, help="right-hand sides per product (single-matrix workloads)")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--configs", default="auto",
                    help="extra configuration sections in the line: laplace, eigen, batch (comma list), all, none; "
                         "auto = all for the default 280^3 headline, none otherwise")
    ap.add_argument("--no-probes", action="store_true", help="skip the FP64 / random-read probes (unit-count roofs)")
    ap.add_argument("--prefetch", type=int, default=None,
                    help="L2 prefetch distance of the timed plan (default: the plan's own choice)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--batch-config", default=None,
                    help="item_nnz,schedule,ctas_per_sm of the batched launch instead of the autotuner's choice")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer measurement")
    ap.add_argument("--no-forms", action="store_true", help="skip the comparison of forms")
    ap.add_argument("--forms", default="all",
                    help="comma list of form groups to run: variants, sym, spmm, solver, ordering, block (or all)")
    ap.add_argument("--form-steps", type=int, default=100, help="timed steps per kernel in the ordering forms")
    ap.add_argument("--selector", action="store_true",
                    help="train the cost model on generated matrices (seeds >= 1000) and report its choice, "
                         "its regret against the exhaustive sweep and its gain over the default")
    ap.add_argument("--selector-train", type=int, default=100, help="training matrices for --selector")
    ap.add_argument("--selector-stride", type=int, default=4,
                    help="batch workload: sweep every n-th member exhaustively for the regret")
    return ap.parse_args()


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def load_workload(name):
    import gen
    if name.startswith("poisson3d_"):
        A = gen.poisson3d_var(int(name.split("_")[1]), seed=0)
    elif name == "eigen_6201600":
        A = gen.eigen_shaped(6_201_600, seed=0)
    elif name == "laplace2d_256":
        A = gen.laplace2d(256)
    else:
        raise ValueError(name)
    return A


def measured_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_fingerprint(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1101_0091_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {"crs_l1": ["k_lanes.cu", "device.cuh", "layout.h"],
                  "crs_staged": ["k_staged.cu", "device.cuh", "layout.h"],
                  "sell": ["k_sell.cu", "device.cuh", "layout.h"],
                  "sym": ["k_sym.cu", "device.cuh", "layout.h"],
                  "batch": ["batch_kernel.cuh", "batch.cu", "device.cuh", "layout.h"]}


def ncu_record(kernel: str, workload: str) -> dict:
    """The committed ncu record of a kernel on a workload, if it was taken on the
    current kernel sources (else {})."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return {}
    with open(p) as f:
        e = json.load(f).get(f"{kernel}/{workload}")
    src = KERNEL_SOURCES.get(kernel.split("_s")[0] if kernel.startswith("sell") else kernel)
    if not e or not src or e.get("source_fingerprint") != kernel_fingerprint(src):
        return {}
    return e


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{kernel}/{workload}")
    src = KERNEL_SOURCES.get(kernel.split("_s")[0] if kernel.startswith("sell") else kernel)
    if not e or not src or e.get("source_fingerprint") != kernel_fingerprint(src):
        return None
    return e.get("dram_bytes_per_launch")


def dram_view(traffic, bytes_min, nnz, kern_s, hbm, pm) -> dict:
    """From the recorded ncu DRAM bytes of the kernel: DRAM GB/s over the
    measured launch time, its fraction of the copy peak, and kappa_gpu =
    (DRAM bytes - V_min) / nnz."""
    if traffic is None:
        return {"dram_gbs": None, "dram_frac": None, "kappa_gpu": None}
    return {"dram_gbs": round(traffic / kern_s / 1e9, 1), "dram_frac": round(traffic / kern_s / 1e9 / hbm, 4),
            "kappa_gpu": round(pm.kappa_gpu(traffic, bytes_min, nnz), 4)}


# Host-side baselines of the headline, run after every GPU section of the line:
# run before the sections, these host runs lowered the batch section's
# end-to-end figure (host copies) from 126 to 90-96 GFlop/s.
LATE_HOST_WORK = []


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons; summary() keeps
    the samples taken inside [t0, t1] (host wall clock)."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self, t0: float, t1: float):
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                if not (t0 - 0.05 <= ts <= t1 + 0.05):
                    continue
                sm.append(float(f[2]))
                mx.append(float(f[3]))
                pw.append(float(f[4]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "power_w_median": statistics.median(pw),
                "reasons": sorted(reasons), "samples": len(sm)}


def time_oracle(fn, steps: int, budget_s: float):
    fn()
    ts = []
    t_end = time.perf_counter() + budget_s
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        fn()
        ts.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end:
            break
    return ts


def batch_members(count):
    import gen
    As = [gen.powerlaw_batch_member(m) for m in range(count)]
    Bs = [gen.rhs_block(A.n_cols, 4, seed=0, stream=2 * m + 1) for m, A in enumerate(As)]
    return As, Bs


def reference_arm(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import gen
    import oracle
    if args.workload.startswith("powerlaw_batch"):
        As, Bs = batch_members(args.batch_count)
        flops = sum(8 * A.nnz for A in As)
        fn = lambda: [oracle.spmm(A, B) for A, B in zip(As, Bs)]  # noqa: E731
        sample = f"all {len(As)} members, k=4, single-threaded FP64 oracle loop"
    else:
        A = load_workload(args.workload)
        B = gen.uniform(A.n_cols, seed=0)
        flops = 2 * A.nnz
        fn = lambda: oracle.spmv(A, B)  # noqa: E731
        sample = "full product, single-threaded FP64 oracle loop"
    ts = time_oracle(fn, max(1, min(args.steps, 20)), budget_s=90.0)
    t = sum(ts) / len(ts)
    value = flops / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GFlop/s", "n_gpus": args.gpus,
            "steps": len(ts), "warmup": 1, "ms_per_step": round(t * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload]},
            "cpu_baseline": {"value": round(value, 4), "unit": "GFlop/s", "cores": 1, "kind": "oracle",
                             "sample": f"{sample}, {len(ts)} timed runs"},
            "e2e": {"value": round(value, 4), "unit": "GFlop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def all_max(values, world: int):
    """Element-wise maximum over ranks (replicas: the slowest rank sets the
    time).  CUDA tensors under NCCL, CPU tensors under gloo."""
    if world <= 1:
        return list(values)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu().tolist()]


def replica_value(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Whole-job throughput of N independent replicas: all ranks' units over the
    slowest rank's time."""
    return units_per_rank * world / seconds_max


SLOWDOWN_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(c) -> bool:
    """A timed region that saw a hardware or thermal slowdown, or SM clocks
    well below their maximum with no reason given (a clock lock left by
    someone), is not a valid measurement; sw_power_cap alone is kept."""
    if not c or not c.get("samples"):
        return False
    if any(r in c.get("reasons", []) for r in SLOWDOWN_REASONS):
        return True
    return bool(c.get("sm_mhz") and c.get("sm_max_mhz") and c["sm_mhz"] < 0.9 * c["sm_max_mhz"]
                and not c.get("reasons"))


class Timer:
    """CUDA-event timing of `steps` calls on one stream, with a barrier and a
    synchronize on both sides and nvidia-smi clock samples inside the region."""

    def __init__(self, torch, stream, world, local):
        self.torch, self.stream, self.world, self.local = torch, stream, world, local

    def barrier(self):
        self.torch.cuda.synchronize()
        if self.world > 1:
            self.torch.distributed.barrier()
            self.torch.cuda.synchronize()

    def run(self, fn, steps, warmup, sample_clocks=False):
        torch = self.torch
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        clk = ClockSampler(self.local) if sample_clocks else None
        if clk:
            clk.__enter__()
        t_warm = time.perf_counter() + (0.8 if clk else 0.0)
        i = 0
        while i < warmup or time.perf_counter() < t_warm:   # warm-up; also lets the sampler start
            fn()
            i += 1
            if i % 50 == 0:
                self.stream.synchronize()
        self.barrier()
        t0 = time.time()
        ev[0].record(self.stream)
        for s in range(steps):
            fn()
            ev[s + 1].record(self.stream)
        self.stream.synchronize()
        t1 = time.time()
        self.barrier()
        if clk:
            clk.__exit__(None, None, None)
        per = [ev[s].elapsed_time(ev[s + 1]) for s in range(steps)]
        total_ms = all_max([ev[0].elapsed_time(ev[-1])], self.world)[0]
        return {"total_ms": total_ms, "per_ms": per, "wall_s": t1 - t0,
                "clocks": clk.summary(t0, t1) if clk else None}

    def run_checked(self, fn, steps, warmup):
        """run() with clock samples; a region whose clocks are rejected (on
        any rank) is measured once more, and the line keeps the first
        region's clock record beside the second."""
        r = self.run(fn, steps, warmup, sample_clocks=True)
        if all_max([1.0 if clocks_rejected(r["clocks"]) else 0.0], self.world)[0] > 0:
            first = r["clocks"]
            r = self.run(fn, steps, warmup, sample_clocks=True)
            r["clocks"] = dict(r["clocks"] or {}, remeasured_after=first)
        return r


def single_workload(args, torch, spmv, pm, timer, stream, world, rank):
    import gen
    A = load_workload(args.workload)
    k = args.k
    Bh = gen.uniform(A.n_cols, seed=0) if k == 1 else gen.rhs_block(A.n_cols, k, seed=0)
    vid, sigma = VARIANTS[args.variant]
    plan = spmv.Plan.from_csr(A, variant=vid, sell_sigma=sigma, val_fp32=args.fp32_val)
    if args.prefetch is not None:
        plan.set_tuning(prefetch_distance=args.prefetch)
    B = torch.from_numpy(Bh).cuda()
    C = torch.empty((A.n_rows,) if k == 1 else (A.n_rows, k), dtype=torch.float64, device="cuda")
    stream.wait_stream(torch.cuda.current_stream())
    fn = (lambda: plan.apply(B, C, stream)) if k == 1 else (lambda: plan.apply_block(B, C, k, stream))
    tr = pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz, k=k, val_bytes=4 if args.fp32_val else 8)
    if vid == spmv.SPMV_SYM:
        tr = pm.gpu_sym_min_traffic(A.n_rows, A.nnz, plan.info().sym_nnz, k=k, val_bytes=4 if args.fp32_val else 8)
    r = timer.run_checked(fn, args.steps, args.warmup)
    plan.check(stream)
    t_step = r["total_ms"] / 1e3 / args.steps
    kern_s = statistics.mean(r["per_ms"]) / 1e3
    hbm, hbm_kind = measured_hbm()
    achieved = tr.bytes_min / kern_s / 1e9
    kname = "sell" if args.variant.startswith("sell") else args.variant
    line = {
        "metric": METRIC, "value": round(replica_value(tr.flops, t_step, world) / 1e9, 3), "unit": "GFlop/s",
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_step * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload], "kernel": args.variant,
                   "prefetch_distance": plan.tuning().prefetch_distance,
                   "val_storage": "f32" if args.fp32_val else "f64", "k": k, "n_rows": A.n_rows, "nnz": A.nnz,
                   "l2": (f"inputs larger than L2 ({tr.bytes_min / 1e9:.2f} GB vs 129 MB), no flush"
                          if tr.bytes_min > 2 * 129e6 else "inputs L2-resident (warm figure)"),
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "hbm_gbs": round(achieved, 1),
        "roofline": dict({"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                          "frac": round(achieved / hbm, 4), "peak_kind": hbm_kind,
                          "traffic": ncu_traffic(kname, args.workload),
                          "algorithmic_bytes_per_launch": tr.bytes_min,
                          "frac_of_nominal_7900": round(achieved / 7900.0, 4),
                          "fp64_frac": round(tr.flops / kern_s / 1e9 / fp64_peak(), 4)},
                         **dram_view(ncu_traffic(kname, args.workload), tr.bytes_min, A.nnz, kern_s, hbm, pm)),
        "gpu_launches": args.steps,
        "clocks": r["clocks"],
        "wall_s_timed": round(r["wall_s"], 4),
        "paper_context": PAPER_CONTEXT,
    }
    if not args.no_e2e:
        # through the C ABI from pinned host buffers: every step copies its B in (H2D) and its C out (D2H)
        # inside the timed region.  Pipelined steps (spmv_apply_host_async: copy-in of step i+1 and
        # copy-out of step i-1 overlap the product of step i), and one synchronous call per step.
        Bpin = [torch.from_numpy(np.ascontiguousarray(Bh)).pin_memory() for _ in range(2)]
        Cpin = [torch.empty(C.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
        n_e2e = max(3, min(args.steps, 40))
        for i in range(4):
            plan.apply_host_async(Bpin[i % 2], Cpin[i % 2], k, stream)
        plan.host_sync()
        timer.barrier()
        t0 = time.perf_counter()
        for i in range(n_e2e):
            plan.apply_host_async(Bpin[i % 2], Cpin[i % 2], k, stream)
        plan.host_sync()
        e2e_t = (time.perf_counter() - t0) / n_e2e
        t0 = time.perf_counter()
        for _ in range(5):
            plan.apply_host_ptr(Bpin[0].data_ptr(), k, Cpin[0].data_ptr(), stream)
        sync_t = (time.perf_counter() - t0) / 5
        e2e_t, sync_t = all_max([e2e_t, sync_t], world)
        line["e2e"] = {"value": round(tr.flops * world / e2e_t / 1e9, 3), "unit": "GFlop/s",
                       "h2d_bytes_per_step": 8 * A.n_cols * k, "d2h_bytes_per_step": 8 * A.n_rows * k,
                       "api": "spmv_apply_host_async, pipelined, host_sync at the end",
                       "synchronous_call_gflops": round(tr.flops * world / sync_t / 1e9, 3)}
    groups = set() if args.no_forms else (
        {"variants", "sym", "spmm", "solver", "ordering", "block"} if args.forms == "all" else set(args.forms.split(",")))
    poisson, eigen = args.workload.startswith("poisson3d"), args.workload.startswith("eigen")
    if "variants" in groups and poisson:
        line["forms"] = poisson_forms(A, Bh, torch, spmv, pm, timer, stream, plan, B, C)
    if "sym" in groups and k == 1 and (poisson or eigen):
        line.setdefault("forms", {}).update(sym_forms(A, torch, spmv, pm, timer, stream, B, C))
    if "spmm" in groups and k == 1 and (poisson or eigen):
        line["spmm"] = spmm_forms(A, torch, spmv, pm, timer, stream,
                                  ("crs_l1", "crs_staged", "sell_s256") if poisson else
                                  ("crs_l1", "sell_s256", "sell_s4096"))
    if "solver" in groups and k == 1 and poisson:
        line["solver"] = cg_forms(A, torch, spmv, pm, stream)
    if "solver" in groups and k == 1 and eigen:
        line["solver"] = lanczos_forms(A, torch, spmv, pm, stream)
    if "ordering" in groups and k == 1 and eigen:
        line["ordering"] = ordering_forms(A, torch, spmv, pm, timer, stream, B, C, args.workload, args.form_steps)
    if "block" in groups and args.workload == "laplace2d_256":
        line["forms"] = laplace_section(torch, spmv, pm, stream, with_cpu=False)
    if args.selector:
        line["selector"] = plan_selector(args, A, timer, stream, tr, spmv)
    if rank == 0 and not args.no_cpu:
        def cpu_baselines():
            import oracle
            ts = time_oracle(lambda: oracle.spmv(A, Bh) if k == 1 else oracle.spmm(A, Bh), 3, budget_s=30.0)
            line["cpu_baseline"] = {"value": round(tr.flops / min(ts) / 1e9, 4), "unit": "GFlop/s", "cores": 1,
                                    "host_cores": os.cpu_count(),
                                    "kind": "oracle", "sample": f"full product, best of {len(ts)} single-threaded runs"}
            import baselines
            if baselines.available() and k == 1:
                baselines.spmv(A, Bh)  # warm-up (first touch, thread start)
                tn = time_oracle(lambda: baselines.spmv(A, Bh), 5, budget_s=15.0)
                line["cpu_node_baseline"] = {
                    "value": round(tr.flops / min(tn) / 1e9, 4), "unit": "GFlop/s", "cores": baselines.threads(),
                    "kind": "OpenMP row-parallel CRS loop (the paper's node-level scheme), same arithmetic as the "
                            "oracle",
                    "sample": f"full product, best of {len(tn)}",
                    "gpu_over_cpu_node": round(line["value"] / world / (tr.flops / min(tn) / 1e9), 1)}
        LATE_HOST_WORK.append(cpu_baselines)
    plan.close()
    return line


def poisson_forms(A, Bh, torch, spmv, pm, timer, stream, plan, B, C):
    """Chosen forms vs plain CRS on the same matrix (median event time of 200 steps)."""
    forms = {}
    tr = pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz)

    def med(fn, steps=200):
        return statistics.median(timer.run(fn, steps, 10)["per_ms"]) / 1e3

    for name in ("crs_l1", "crs_staged", "sell_s256"):
        vid, sigma = VARIANTS[name]
        plan.set_variant(vid, sigma)
        t = med(lambda: plan.apply(B, C, stream))
        forms[name] = {"gflops": round(tr.flops / t / 1e9, 1), "hbm_gbs": round(tr.bytes_min / t / 1e9, 1)}
    plan.set_variant(*VARIANTS["crs_l1"])
    # cold figure: L2 flushed (a write of 2 x the L2 size) before every timed launch
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    flush = torch.empty(2 * l2, dtype=torch.uint8, device="cuda")
    cold = []
    for i in range(25):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.apply(B, C, stream)
        e1.record(stream)
        stream.synchronize()
        if i >= 5:
            cold.append(e0.elapsed_time(e1) / 1e3)
    t_cold = statistics.median(cold)
    forms["crs_l1_cold"] = {"gflops": round(tr.flops / t_cold / 1e9, 1), "hbm_gbs": round(tr.bytes_min / t_cold / 1e9, 1),
                            "flush_bytes": 2 * l2, "note": "L2 flushed before each launch; the row above is warm"}
    del flush
    with spmv.Plan.from_csr(A, val_fp32=True) as p32:
        t = med(lambda: p32.apply(B, C, stream))
        tr32 = pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz, val_bytes=4)
        hbm, _ = measured_hbm()
        # 8 streamed bytes per entry instead of 12, and one FP64 FMA per entry: both roofs are close
        t_b = max(tr32.bytes_min / (hbm * 1e9), tr.flops / (fp64_peak() * 1e9))
        forms["crs_l1_fp32val"] = {"gflops": round(tr.flops / t / 1e9, 1),
                                   "hbm_gbs": round(tr32.bytes_min / t / 1e9, 1), "err_bound": "2e-7*sum|ab|",
                                   "bound": "max(HBM time of V_min with 4-byte values, FP64 time of the FMAs)",
                                   "bound_gflops": round(tr.flops / t_b / 1e9, 1), "frac_of_bound": round(t_b / t, 4)}
    # local/halo split: last 10% of the columns copied from pinned host memory on a side stream
    h = A.n_cols - A.n_cols // 10
    with spmv.Plan.from_csr(A, halo_begin=h) as ps:
        halo = torch.from_numpy(Bh[h:].copy()).pin_memory()
        cs = torch.cuda.Stream()
        t_ov = med(lambda: ps.apply_split(B, halo, C, stream, cs), 100)
        t_ser = med(lambda: ps.apply_split(B, halo, C, stream, stream), 100)
        info = ps.info()
        hbm, _ = measured_hbm()
        # the split's own bound: V_min plus the halo pass's extra bytes at the copy peak
        t_bound = (tr.bytes_min + pm.gpu_split_extra_bytes(info.n_halo_rows)) / (hbm * 1e9)
        forms["split_overlapped"] = {"gflops": round(tr.flops / t_ov / 1e9, 1), "ms": round(t_ov * 1e3, 4),
                                     "halo_bytes_h2d": 8 * (A.n_cols - h), "n_halo_rows": info.n_halo_rows,
                                     "bound_gflops": round(tr.flops / t_bound / 1e9, 1),
                                     "frac_of_bound": round(t_bound / t_ov, 4)}
        forms["split_serial_copy"] = {"gflops": round(tr.flops / t_ser / 1e9, 1), "ms": round(t_ser * 1e3, 4)}
        forms["split_penalty_eq2_model"] = round(pm.split_penalty(A.nnz / A.n_rows), 4)
    return forms


def sym_forms(A, torch, spmv, pm, timer, stream, B, C):
    """Symmetric CRS (Sec. 1.3.1) on the same matrix: the stored triangle, C
    zeroed and mirrors added atomically; median event time of 200 steps (the
    zeroing is inside the timed region).  GFlop/s count the full product's
    flops; hbm_gbs counts the triangle's V_min."""
    out = {}
    for f32 in (False, True):
        with spmv.Plan.from_csr(A, variant=spmv.SPMV_SYM, val_fp32=f32) as p:
            t = statistics.median(timer.run(lambda: p.apply(B, C, stream), 200, 10)["per_ms"]) / 1e3
            tr = pm.gpu_sym_min_traffic(A.n_rows, A.nnz, p.info().sym_nnz, val_bytes=4 if f32 else 8)
            out["sym_fp32val" if f32 else "sym"] = {
                "gflops": round(tr.flops / t / 1e9, 1), "hbm_gbs": round(tr.bytes_min / t / 1e9, 1),
                "us": round(t * 1e6, 2), "stored_entries": p.info().sym_nnz}
    return out


def spmm_forms(A, torch, spmv, pm, timer, stream, names):
    """k right-hand sides on the full matrix (a11): median event time per
    product for the named kernels.  Each nonzero needs k FP64 FMAs, so for
    k >= 2 the bound is the FP64 pipe (2k nnz flops at 1258.6 GFLOP/s), not
    HBM."""
    import gen
    hbm, _ = measured_hbm()
    out = {"bound": "max(V_min(k) / measured copy peak, 2 k nnz / FP64 peak)"}
    with spmv.Plan.from_csr(A) as p:
        for k in (2, 4, 8, 16):
            B = torch.from_numpy(gen.rhs_block(A.n_cols, k, seed=0)).cuda()
            C = torch.empty_like(B)
            stream.wait_stream(torch.cuda.current_stream())
            tr = pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz, k=k)
            t_bound = max(tr.bytes_min / (hbm * 1e9), tr.flops / (fp64_peak() * 1e9))
            row = {"bound_us": round(t_bound * 1e6, 1)}
            for name in names:
                vid, sigma = VARIANTS[name]
                p.set_variant(vid, sigma)
                t = statistics.median(timer.run(lambda: p.apply_block(B, C, k, stream), 30, 3)["per_ms"]) / 1e3
                row[name] = {"us": round(t * 1e6, 1), "gflops": round(tr.flops / t / 1e9, 1),
                             "fp64_frac": round(tr.flops / t / 1e9 / fp64_peak(), 4),
                             "frac_of_bound": round(t_bound / t, 4)}
            out[f"k{k}"] = row
            del B, C
    return out


def ordering_forms(A, torch, spmv, pm, timer, stream, B, C, workload, steps=100):
    """The same matrix in three numberings (Sec. 1.3.1): as generated (the
    HMeP-like numbering), renumbered by the 400 x 15,504 Kronecker transpose
    (HMEp-like) and reordered by RCM.  Per numbering: bandwidth, mean |i - j|,
    and median event times of SELL-32-4096 and CRS_L1; for RCM also the host
    time of the permutation and the device time of moving B in and C out.
    kappa_gpu = (DRAM bytes - V_min) / nnz where an ncu capture of that
    numbering is recorded in profiles/traffic.json."""
    import gen
    tr = pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz)
    rows = np.repeat(np.arange(A.n_rows, dtype=np.int64), np.diff(A.row_ptr))
    out = {}
    t0 = time.perf_counter()
    rcm_perm = spmv.rcm(A.n_rows, A.row_ptr, A.col_idx)
    t_rcm = time.perf_counter() - t0
    orders = [("natural", None), ("kronecker_transposed", gen.kronecker_transpose(400, A.n_rows // 400)),
              ("rcm", rcm_perm)]
    for name, perm in orders:
        if perm is None:
            rp, ci, va = A.row_ptr, A.col_idx, A.val
        else:
            rp, ci, va = spmv.permute_csr(A.n_rows, A.row_ptr, A.col_idx, A.val, perm)
        d = np.abs(rows - ci.astype(np.int64))
        row = {"bandwidth": int(d.max()), "mean_abs_i_minus_j": round(float(d.mean()), 1)}
        with spmv.Plan(A.n_rows, A.n_cols, rp, ci, va, variant=spmv.SPMV_SELL, sell_sigma=4096) as p:
            for vname, vid, sigma in (("sell_s4096", spmv.SPMV_SELL, 4096), ("crs_l1", spmv.SPMV_CRS_L1, 1)):
                p.set_variant(vid, sigma)
                t = statistics.median(timer.run(lambda: p.apply(B, C, stream), steps, 3)["per_ms"]) / 1e3
                key = ("sell" if vname.startswith("sell") else vname)
                dram = ncu_traffic(key, f"{workload}:{name}")
                row[vname] = {"us": round(t * 1e6, 1), "gflops": round(tr.flops / t / 1e9, 1),
                              "hbm_gbs": round(tr.bytes_min / t / 1e9, 1),
                              "kappa_gpu": (round(pm.kappa_gpu(dram, tr.bytes_min, A.nnz), 3)
                                            if dram is not None else None)}
        if perm is not None and name == "rcm":
            with spmv.Reorder(perm) as r:
                Bp, Cp = torch.empty_like(B), torch.empty_like(C)
                t_g = statistics.median(timer.run(lambda: r.gather(B, Bp, stream), steps, 3)["per_ms"]) / 1e3
                t_s = statistics.median(timer.run(lambda: r.scatter(Cp, C, stream), steps, 3)["per_ms"]) / 1e3
            row["host_rcm_s"] = round(t_rcm, 2)
            row["gather_B_us"] = round(t_g * 1e6, 1)
            row["scatter_C_us"] = round(t_s * 1e6, 1)
        out[name] = row
    return out


def cg_bytes_per_iteration(pm, A, k: int) -> int:
    """Algorithmic bytes of one CG iteration of the library: the SpMM's V_min
    (P read, Q written) + alpha (read P, Q) + update (read X, P, R, Q; write
    X, R) + direction (read R, P; write P): V_min + 88 k n bytes."""
    return pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz, k=k).bytes_min + 88 * k * A.n_rows


def cg_forms(A, torch, spmv, pm, stream, iters: int = 50):
    """Conjugate gradients on k columns through the default plan, a fixed
    number of iterations (rtol = 0), polled once: time per iteration, the
    solver's flop rate (SpMM + 10 k n vector flops per iteration) and its
    algorithmic bytes against the measured copy peak."""
    import gen
    hbm, hbm_kind = measured_hbm()
    out = {"method": "CG (Hestenes-Stiefel), k independent columns, graph-replayed iterations",
           "iterations": iters,
           "bound": "SpMM at max(HBM, FP64-pipe) time of its V_min and 2k nnz flops, plus the vector "
                    "kernels' 88 k n bytes at the measured copy peak (the kernels run one after another)"}
    for k in (1, 4, 8, 16):
        # k = 1 is HBM-bound; k >= 2 is FP64-pipe-bound, where CRS_L1 runs its column-split form
        with spmv.Plan.from_csr(A, variant=spmv.SPMV_CRS_L1) as p:
            B = torch.from_numpy(gen.rhs_block(A.n_cols, k, seed=0)).cuda()
            X = torch.zeros_like(B)
            stream.wait_stream(torch.cuda.current_stream())
            with spmv.Solver(p, k) as s:
                s.cg(B, X, max_iter=3, rtol=0.0, check_every=iters, stream=stream)  # warm-up
                ts = []
                for _ in range(3):
                    X.zero_()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    it, rr, summ = s.cg(B, X, max_iter=iters, rtol=0.0, check_every=iters, stream=stream)
                    ts.append(time.perf_counter() - t0)
        t_it = min(ts) / iters
        flops = 2 * k * A.nnz + 10 * k * A.n_rows
        byts = cg_bytes_per_iteration(pm, A, k)
        spmm = pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz, k=k)
        t_bound = (max(spmm.bytes_min / (hbm * 1e9), spmm.flops / (fp64_peak() * 1e9))
                   + 88 * k * A.n_rows / (hbm * 1e9))
        out[f"k{k}"] = {"plan_variant": "crs_l1",
                        "us_per_iteration": round(t_it * 1e6, 1), "gflops": round(flops / t_it / 1e9, 1),
                        "hbm_gbs": round(byts / t_it / 1e9, 1), "bytes_per_iteration": byts,
                        "bound_us": round(t_bound * 1e6, 1), "frac_of_bound": round(t_bound / t_it, 4),
                        "column_iterations_per_s": round(k / t_it, 1)}
    out["hbm_peak"] = hbm
    out["fp64_peak_gflops"] = round(fp64_peak(), 1)
    out["timing"] = "host wall clock around the synchronous solve (one poll at the end), best of 3"
    return out


def lanczos_forms(A, torch, spmv, pm, stream, m: int = 30):
    """Lanczos (no reorthogonalisation) on k start vectors through the
    selector's SELL-32-4096 plan: time per step.  Bytes per step: V_min(k) +
    alpha (read W, v, v_prev; write W) + beta (read W, v; write W) + scale
    (read W; write v) = V_min + 72 k n."""
    import gen
    hbm, _ = measured_hbm()
    out = {"method": "Lanczos three-term recurrence, k independent start vectors", "steps": m}
    with spmv.Plan.from_csr(A, variant=spmv.SPMV_SELL, sell_sigma=4096) as p:
        for k in (1, 4, 16):
            V0 = torch.from_numpy(gen.rhs_block(A.n_cols, k, seed=0)).cuda()
            stream.wait_stream(torch.cuda.current_stream())
            with spmv.Solver(p, k) as s:
                s.lanczos(V0, 3, stream=stream)
                ts = []
                for _ in range(3):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    s.lanczos(V0, m, stream=stream)
                    ts.append(time.perf_counter() - t0)
            t_it = min(ts) / m
            spmm = pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz, k=k)
            byts = spmm.bytes_min + 72 * k * A.n_rows
            t_bound = (max(spmm.bytes_min / (hbm * 1e9), spmm.flops / (fp64_peak() * 1e9))
                       + 72 * k * A.n_rows / (hbm * 1e9))
            out[f"k{k}"] = {"us_per_step": round(t_it * 1e6, 1),
                            "gflops": round((2 * k * A.nnz + 8 * k * A.n_rows) / t_it / 1e9, 1),
                            "hbm_gbs": round(byts / t_it / 1e9, 1), "bound_us": round(t_bound * 1e6, 1),
                            "frac_of_bound": round(t_bound / t_it, 4)}
    out["note"] = ("at k = 1 the random gathers of this matrix make its SpMM L2-bound (SELL-32-4096 reaches "
                   "about 0.55 of the copy peak alone), so the HBM/FP64 bound is not reachable there")
    return out


def laplace_section(torch, spmv, pm, stream, with_cpu: bool = True) -> dict:
    """The 2D 5-point Laplacian on 256^2 (65,536 rows, 326,656 nonzeros; the
    first configuration) and its k in {1, 4, 8, 16} right-hand sides with
    FP64 and FP32-stored values (the precision / block configuration).  The
    5 MB matrix is L2-resident, so one product is latency- and launch-bound;
    per (k, storage) four device times are reported:
      isolated: one launch between two events, queue empty before it;
      back_to_back: 200 launches between two events (launch gaps included);
      graph: 100 products captured into one CUDA graph, replayed (the
             kernel's own latency, launch overhead taken off the host);
      cold: one launch after a 256 MB write has flushed L2.
    Errors per right-hand-side column against the oracle's CRS loop (FP64
    values; the FP32-value form also against the oracle's FP32-value loop),
    as the largest |y - y_ref| / (tol * sum_j |a_ij b_j|) of the column."""
    import gen
    import oracle
    A = gen.laplace2d(256)
    hbm, _ = measured_hbm()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {"workload": "laplace2d_256", "description": WORKLOADS["laplace2d_256"], "n_rows": A.n_rows,
           "nnz": A.nnz, "timing": "median CUDA-event times (see keys); GFlop/s = 2 k nnz / time",
           "err_bound": {"f64val": "1e-13*sum|ab| vs the FP64 oracle", "f32val": "2e-7*sum|ab| vs the FP64 oracle"}}

    def ev_pair():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    for f32 in (False, True):
        with spmv.Plan.from_csr(A, val_fp32=f32) as p:
            for k in (1, 4, 8, 16):
                Bh = gen.uniform(A.n_cols, seed=0) if k == 1 else gen.rhs_block(A.n_cols, k, seed=0)
                B = torch.from_numpy(Bh).cuda()
                C = torch.empty((A.n_rows,) if k == 1 else (A.n_rows, k), dtype=torch.float64, device="cuda")
                stream.wait_stream(torch.cuda.current_stream())

                def fn(st=stream):
                    (p.apply(B, C, st) if k == 1 else p.apply_block(B, C, k, st))
                iso, cold = [], []
                for i in range(60):
                    if i % 2:
                        with torch.cuda.stream(stream):
                            flush.zero_()
                    else:
                        stream.synchronize()
                    e0, e1 = ev_pair()
                    e0.record(stream)
                    fn()
                    e1.record(stream)
                    stream.synchronize()
                    (cold if i % 2 else iso).append(e0.elapsed_time(e1) / 1e3)
                e0, e1 = ev_pair()
                e0.record(stream)
                for _ in range(200):
                    fn()
                e1.record(stream)
                stream.synchronize()
                b2b = e0.elapsed_time(e1) / 1e3 / 200
                # 100 products in one CUDA graph, captured on a side stream
                g = torch.cuda.CUDAGraph()
                cap = torch.cuda.Stream()
                cap.wait_stream(torch.cuda.current_stream())
                with torch.cuda.graph(g, stream=cap, capture_error_mode="thread_local"):
                    for _ in range(100):
                        fn(torch.cuda.current_stream())
                torch.cuda.synchronize()
                gts = []
                for _ in range(7):
                    e0, e1 = ev_pair()
                    e0.record(stream)
                    with torch.cuda.stream(stream):
                        g.replay()
                    e1.record(stream)
                    stream.synchronize()
                    gts.append(e0.elapsed_time(e1) / 1e3 / 100)
                del g
                y = C.cpu().numpy()
                B2 = Bh.reshape(A.n_cols, k)
                y2 = y.reshape(A.n_rows, k)
                ref = oracle.spmm(A, B2)
                scale = oracle.abs_scale(A, B2)
                tol = 2e-7 if f32 else 1e-13
                col_err = [oracle.max_err_ratio(y2[:, c], ref[:, c], scale[:, c], tol) for c in range(k)]
                row = {}
                if f32:
                    ref32 = oracle.spmm(A, B2, f32val=True)
                    row["err_ratio_vs_f32val_oracle_at_1e-13"] = round(max(
                        oracle.max_err_ratio(y2[:, c], ref32[:, c], scale[:, c], 1e-13) for c in range(k)), 6)
                tr = pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz, k=k, val_bytes=4 if f32 else 8)
                ti, tc, tg = statistics.median(iso[5:]), statistics.median(cold[5:]), statistics.median(gts)
                row.update({
                    "isolated_us": round(ti * 1e6, 2), "isolated_gflops": round(tr.flops / ti / 1e9, 1),
                    "back_to_back_us": round(b2b * 1e6, 2), "back_to_back_gflops": round(tr.flops / b2b / 1e9, 1),
                    "graph_us": round(tg * 1e6, 2), "graph_gflops": round(tr.flops / tg / 1e9, 1),
                    "cold_us": round(tc * 1e6, 2), "cold_gflops": round(tr.flops / tc / 1e9, 1),
                    "cold_hbm_gbs": round(tr.bytes_min / tc / 1e9, 1),
                    "err_ratio_per_column": [round(e, 6) for e in col_err],
                    "bit_identical_columns": int(sum(np.array_equal(y2[:, c], ref[:, c]) for c in range(k)))})
                out[f"k{k}_{'f32' if f32 else 'f64'}val"] = row
    best = min(v["graph_us"] for key, v in out.items() if key.startswith("k1_"))
    out["roofline"] = {"bound": "latency", "note": "L2-resident: the HBM time of V_min is "
                       f"{pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz).bytes_min / (hbm * 1e9) * 1e6:.2f} us, far "
                       "below a kernel's launch-to-finish latency", "graph_us_k1": best}
    if with_cpu:
        Bh = gen.uniform(A.n_cols, seed=0)
        ts = time_oracle(lambda: oracle.spmv(A, Bh), 20, budget_s=5.0)
        out["cpu_baseline"] = {"value": round(2 * A.nnz / min(ts) / 1e9, 4), "unit": "GFlop/s", "cores": 1,
                               "kind": "oracle", "sample": f"full k = 1 product, best of {len(ts)}"}
    del flush
    return out


COST_MODEL_DIR = os.path.join(ROOT, "paper_1101_0091_gb300", "cost_models")


def far_entries(A, reach: int = 32) -> int:
    """Stored entries with |i - j| > reach.  A warp's 32 rows read B entries
    inside a window of about 32 around them (8 sectors of 32 bytes), so
    closer entries share sectors; each farther entry needs a 32-byte sector of
    its own, one random read served by L2 at best."""
    rows = np.repeat(np.arange(A.n_rows, dtype=np.int64), np.diff(A.row_ptr).astype(np.int64))
    return int(np.count_nonzero(np.abs(rows - A.col_idx.astype(np.int64)) > reach))


def eigen_section(torch, spmv, pm, timer, stream, steps: int = 50, with_ordering: bool = True,
                  with_cpu: bool = True) -> dict:
    """The eigenproblem-shaped matrix (6,201,600 = 400 x 15,504 rows, about
    13.8 nonzeros per row, ten of them scattered within +-2^20): every plan
    kernel, SELL-32 with sigma in {1, 256, 4096} among them, and the cost
    model's choice, at k = 1 (median event time of `steps` launches).  Two
    roofs: HBM (V_min at the measured copy peak) and the random reads of B
    (one 32-byte sector per scattered entry at the rate spmv_probe_gather
    measures out of an L2-resident buffer)."""
    import gen
    import oracle
    from paper_1101_0091_gb300 import selector as sel
    A = gen.eigen_shaped(6_201_600, seed=0)
    Bh = gen.uniform(A.n_cols, seed=0)
    B = torch.from_numpy(Bh).cuda()
    C = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
    stream.wait_stream(torch.cuda.current_stream())
    hbm, hbm_kind = measured_hbm()
    tr = pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz)
    n_far = far_entries(A)
    req_rate = MACHINE.get("l2_gathers_per_s")
    t_hbm = tr.bytes_min / (hbm * 1e9)
    # requests from the SMs' L1 to L2 that no schedule avoids: one per scattered
    # entry (its 32-byte sector of B is read by nothing else nearby) and one per
    # 128-byte line of the compulsory streams (V_min)
    req_min = n_far + tr.bytes_min / 128
    t_l2 = req_min / req_rate if req_rate else None
    out = {"workload": "eigen_6201600", "description": WORKLOADS["eigen_6201600"], "n_rows": A.n_rows, "nnz": A.nnz,
           "algorithmic_bytes_per_launch": tr.bytes_min, "scattered_entries": n_far,
           "l2_requests_min": int(req_min),
           "hbm_bound_us": round(t_hbm * 1e6, 1),
           "request_bound_us": round(t_l2 * 1e6, 1) if t_l2 else None,
           "request_bound": "(scattered entries + V_min / 128 B) / the probe's random-read rate per SM and clock "
                            "x SMs x max clock",
           "timing": f"median CUDA-event time of {steps} launches, k = 1"}
    times = {}
    with spmv.Plan.from_csr(A) as p:
        out["auto_variant"] = spmv.VARIANT_NAMES[p.info().variant]
        for name, vid, sigma in sel.PLAN_VARIANTS:
            p.set_variant(vid, sigma)
            t = statistics.median(timer.run(lambda: p.apply(B, C, stream), steps, 3)["per_ms"]) / 1e3
            times[name] = t
            out[name] = {"us": round(t * 1e6, 1), "gflops": round(tr.flops / t / 1e9, 1),
                         "hbm_frac": round(t_hbm / t, 4), "request_frac": round(t_l2 / t, 4) if t_l2 else None}
            if name == "sell_s256":
                out[name]["parity_max_err_ratio"] = round(oracle.max_err_ratio(
                    C.cpu().numpy(), oracle.spmv(A, Bh), oracle.abs_scale(A, Bh), 1e-13), 6)
        sweep = np.array([times[v[0]] for v in sel.PLAN_VARIANTS])
        ck = os.path.join(COST_MODEL_DIR, "plan.bin")
        if os.path.exists(ck):
            cm = sel.CostModel.load(ck)
            c = int(cm.select(spmv.features(A, 1))[0][0])
            cm.close()
            name = sel.PLAN_VARIANTS[c][0]
            out["selector"] = {"model": "paper_1101_0091_gb300/cost_models/plan.bin", "chosen": name,
                               "gflops_chosen": out[name]["gflops"],
                               "gflops_default_crs_l1": out["crs_l1"]["gflops"],
                               "best_in_sweep": sel.PLAN_VARIANTS[int(sweep.argmin())][0],
                               "regret": round(float(sweep[c] / sweep.min() - 1), 4)}
    # FP32-stored values (FP64 accumulation) under AUTO: 8 instead of 12 streamed bytes per slot
    with spmv.Plan.from_csr(A, val_fp32=True) as p32:
        t32 = statistics.median(timer.run(lambda: p32.apply(B, C, stream), steps, 3)["per_ms"]) / 1e3
        y32 = C.cpu().numpy()
        scale = oracle.abs_scale(A, Bh)
        tr32 = pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz, val_bytes=4)
        out["auto_fp32val"] = {
            "variant": spmv.VARIANT_NAMES[p32.info().variant], "us": round(t32 * 1e6, 1),
            "gflops": round(tr.flops / t32 / 1e9, 1), "hbm_gbs": round(tr32.bytes_min / t32 / 1e9, 1),
            "err_ratio_vs_f64_oracle_at_2e-7": round(oracle.max_err_ratio(y32, oracle.spmv(A, Bh), scale, 2e-7), 4),
            "err_ratio_vs_f32val_oracle_at_1e-13": round(oracle.max_err_ratio(
                y32, oracle.spmm(A, Bh.reshape(-1, 1), f32val=True)[:, 0], scale, 1e-13), 4),
            "over_crs_l1_f64": round(times["crs_l1"] / t32, 3)}
    best = min(times, key=times.get)
    tb = times[best]
    out["roofline"] = {"bound": "l2_requests", "kernel": best, "achieved_us": round(tb * 1e6, 1),
                       "achieved": round(req_min / tb / 1e9, 2) if t_l2 else None, "unit": "1e9 requests/s",
                       "peak": round(req_rate / 1e9, 2) if req_rate else None,
                       "frac": round(t_l2 / tb, 4) if t_l2 else None,
                       "hbm_achieved_gbs": round(tr.bytes_min / tb / 1e9, 1), "hbm_peak": hbm,
                       "hbm_frac": round(t_hbm / tb, 4),
                       "frac_of_max_bound": round(max(t_hbm, t_l2 or 0.0) / tb, 4),
                       "traffic": ncu_traffic("sell", "eigen_6201600")}
    rec = ncu_record("sell", "eigen_6201600")
    if rec.get("l2_requests_per_launch") and req_rate and "sell_s256" in times:
        # all L2 requests of SELL-32-256 (the SMs' and the die-to-die fabric's, one ncu launch)
        # over its time here, against the L2-resident probe's request rate
        ts = times["sell_s256"]
        out["roofline"]["sell_s256_l2_requests"] = {
            "sm": rec["sm_requests_per_launch"], "fabric": rec["fabric_requests_per_launch"],
            "all": rec["l2_requests_per_launch"],
            "rate_per_s": round(rec["l2_requests_per_launch"] / ts / 1e9, 1),
            "frac_of_probe_rate": round(rec["l2_requests_per_launch"] / ts / req_rate, 4)}
    out.update(sym_forms(A, torch, spmv, pm, timer, stream, B, C))
    if with_ordering:
        out["ordering"] = ordering_forms(A, torch, spmv, pm, timer, stream, B, C, "eigen_6201600", steps)
    if with_cpu:
        ts = time_oracle(lambda: oracle.spmv(A, Bh), 3, budget_s=10.0)
        out["cpu_baseline"] = {"value": round(tr.flops / min(ts) / 1e9, 4), "unit": "GFlop/s", "cores": 1,
                               "kind": "oracle", "sample": f"full product, best of {len(ts)}"}
    return out


def mixed_row_bound(As, kern_s, hbm) -> dict:
    """Per-row roofline of an uneven batch (k = 4): a row of L entries needs
    12 L + 68 bytes (val/col, row pointer, its 32-byte C row and a 32-byte B row)
    and 8 L flops, so short rows are HBM-bound and long ones FP64-bound; the
    bound is the sum over rows of the larger of the two times."""
    t = 0.0
    for A in As:
        L = np.diff(A.row_ptr).astype(np.float64)
        t += float(np.maximum((12 * L + 68) / (hbm * 1e9), 8 * L / (fp64_peak() * 1e9)).sum())
    return {"mixed_bound_us": round(t * 1e6, 1), "mixed_frac": round(t / kern_s, 4),
            "mixed_bound_kind": "sum over rows of max(HBM time of 12L+68 B, FP64 time of 8L flops)"}


def random_dram_bound(As, bytes_min, hbm, kern_s, k: int = 4) -> dict:
    """A DRAM bound that counts how B is read: each member's B block (8k bytes
    per column) is fetched from HBM once, in the random order of its columns,
    as 64-byte blocks at the random-read rate the HBM probe measures in this
    run; the rest of V_min streams at the copy peak; the two share DRAM time,
    so their times add."""
    rate = MACHINE.get("dram_gathers_per_s")
    if not rate:
        return {}
    b_bytes = sum(8 * k * A.n_cols for A in As)
    t = (b_bytes / 64) / rate + (bytes_min - b_bytes) / (hbm * 1e9)
    return {"random_dram_bound_us": round(t * 1e6, 1), "random_dram_frac": round(t / kern_s, 4),
            "random_dram_bound_kind": "B blocks as 64-byte random fetches at the probe's HBM random-read rate "
                                      "+ the rest of V_min at the copy peak"}


def batch_workload(args, torch, spmv, pm, timer, stream, world, rank):
    As, Bhs = batch_members(args.batch_count)
    nnz = sum(A.nnz for A in As)
    rows = sum(A.n_rows for A in As)
    flops = 8 * nnz
    plans = [spmv.Plan.from_csr(A) for A in As]
    # every member's B and C is a view of one device allocation per operand (members back to
    # back, each 32-byte aligned), so the host path moves each operand in one copy
    nb, nc = [A.n_cols * 4 for A in As], [A.n_rows * 4 for A in As]
    Bflat = torch.from_numpy(np.concatenate([B.ravel() for B in Bhs])).cuda()
    Cflat = torch.empty(sum(nc), dtype=torch.float64, device="cuda")
    Bs = [v.view(A.n_cols, 4) for v, A in zip(torch.split(Bflat, nb), As)]
    Cs = [v.view(A.n_rows, 4) for v, A in zip(torch.split(Cflat, nc), As)]
    stream.wait_stream(torch.cuda.current_stream())
    batch = spmv.Batch(plans, 4, [spmv.SPMV_BATCH_SORTED] * len(As))
    batch.set_io(Bs, Cs)
    tuned = None
    if args.batch_config:
        it, sc, ct = (int(x) for x in args.batch_config.split(","))
        batch.set_config(item_nnz=it, schedule=sc, ctas_per_sm=ct)
        tuned = {"item_nnz": it, "schedule": ["static", "atomic"][sc], "ctas_per_sm": ct, "source": "--batch-config"}
    elif not args.no_autotune:
        best, times = batch.autotune(stream, reps=3)
        tuned = {"item_nnz": best.item_nnz, "schedule": ["static", "atomic"][best.schedule],
                 "ctas_per_sm": best.ctas_per_sm}
    r = timer.run_checked(lambda: batch.apply(stream), args.steps, args.warmup)
    t_step = r["total_ms"] / 1e3 / args.steps
    kern_s = statistics.mean(r["per_ms"]) / 1e3
    bytes_min = sum(pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz, k=4).bytes_min for A in As)
    hbm, hbm_kind = measured_hbm()
    rand_dram = random_dram_bound(As, bytes_min, hbm, kern_s)
    achieved_gf = flops / kern_s / 1e9
    line = {
        "metric": METRIC, "value": round(replica_value(flops, t_step, world) / 1e9, 3), "unit": "GFlop/s",
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_step * 1e3, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload], "members": len(As),
                   "rows": rows, "nnz": nnz, "k": 4, "kernel": "k_batch (sorted row policy, graph replay)",
                   "autotuned": tuned, "l2": "inputs larger than L2, no flush",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "hbm_gbs": round(bytes_min / kern_s / 1e9, 1),
        "roofline": {"bound": "alu", "achieved": round(achieved_gf, 1), "peak": round(fp64_peak(), 1),
                     "unit": "GFLOP/s", "frac": round(achieved_gf / fp64_peak(), 4),
                     "peak_kind": "FP64 FMA rate, " + MACHINE["fp64_kind"],
                     "traffic": ncu_traffic("batch", args.workload), "algorithmic_bytes_per_launch": bytes_min,
                     "hbm_frac": round(bytes_min / kern_s / 1e9 / hbm, 4), "hbm_peak": hbm, "hbm_peak_kind": hbm_kind,
                     **mixed_row_bound(As, kern_s, hbm), **rand_dram},
        "gpu_launches": args.steps,
        "clocks": r["clocks"],
        "wall_s_timed": round(r["wall_s"], 4),
    }
    if not args.no_e2e:
        # end to end through the C ABI from pinned host buffers: every step copies all members' B in,
        # runs the batched launch and copies all C back.  Pipelined (spmv_batch_apply_host_async: the
        # copy-in of step i+1 and the copy-out of step i-1 overlap step i; two pinned sets alternate),
        # and one synchronous spmv_batch_apply_host per step beside it.
        Bpin_flat = [torch.from_numpy(np.concatenate([B.ravel() for B in Bhs])).pin_memory() for _ in range(2)]
        Cpin_flat = [torch.empty(sum(nc), dtype=torch.float64).pin_memory() for _ in range(2)]
        Bpin = [list(torch.split(x, nb)) for x in Bpin_flat]
        Cpin = [list(torch.split(x, nc)) for x in Cpin_flat]
        n_e2e = 40  # the pipeline's fill and drain (one copy each way) stay a few percent of the region
        for i in range(2):
            batch.apply_host_async(Bpin[i % 2], Cpin[i % 2], stream)
        batch.host_sync()
        timer.barrier()
        t0 = time.perf_counter()
        for i in range(n_e2e):
            batch.apply_host_async(Bpin[i % 2], Cpin[i % 2], stream)
        batch.host_sync()
        e2e_t = (time.perf_counter() - t0) / n_e2e

        def step():
            batch.apply_host(Bpin[0], Cpin[0], stream)
            stream.synchronize()
        step()
        t0 = time.perf_counter()
        for _ in range(3):
            step()
        sync_t = (time.perf_counter() - t0) / 3
        e2e_t, sync_t = all_max([e2e_t, sync_t], world)
        line["e2e"] = {"value": round(flops * world / e2e_t / 1e9, 3), "unit": "GFlop/s",
                       "h2d_bytes_per_step": sum(8 * B.size for B in Bhs),
                       "d2h_bytes_per_step": sum(32 * A.n_rows for A in As),
                       "api": "spmv_batch_apply_host_async, pipelined, host_sync at the end (members back to back: "
                              "one copy per operand and step)",
                       "synchronous_call_gflops": round(flops * world / sync_t / 1e9, 3)}
    if not args.no_forms:
        forms = {}
        def med(fn, steps=20):
            return statistics.median(timer.run(fn, steps, 3)["per_ms"]) / 1e3
        forms["batched_sorted_tuned"] = {"gflops": round(flops / kern_s / 1e9, 1)}
        t = med(lambda: batch.apply_separate(stream), 3)
        forms["separate_launches_plan_default"] = {"gflops": round(flops / t / 1e9, 2), "launches": len(As)}
        for pol in range(spmv.SPMV_BATCH_N_POLICIES - 1):   # every policy but the sorted one timed above
            batch.set_policies([pol] * len(As))
            t = med(lambda: batch.apply(stream))
            forms[f"batched_fixed_{spmv.POLICY_NAMES[pol]}"] = {"gflops": round(flops / t / 1e9, 1)}
        line["forms"] = forms
    if args.selector:
        line["selector"] = batch_selector(args, As, batch, timer, stream, flops, spmv)
    elif os.path.exists(os.path.join(COST_MODEL_DIR, "batch.bin")):
        line["learned_policies"] = batch_learned(As, batch, timer, stream, flops, spmv)
    if rank == 0 and not args.no_cpu:
        import oracle
        sub = min(len(As), 64)
        ts = time_oracle(lambda: [oracle.spmm(A, B) for A, B in zip(As[:sub], Bhs[:sub])], 1, budget_s=30.0)
        fl = sum(8 * A.nnz for A in As[:sub])
        line["cpu_baseline"] = {"value": round(fl / min(ts) / 1e9, 4), "unit": "GFlop/s", "cores": 1,
                                "host_cores": os.cpu_count(),
                                "kind": "oracle", "sample": f"first {sub} members, k=4, best of {len(ts)}"}
    batch.close()
    for p in plans:
        p.close()
    return line


def batch_learned(As, batch, timer, stream, flops, spmv) -> dict:
    """The shipped batch cost model (trained on members timed inside a mixed
    batch) picks each member's row policy, guarded: a member leaves the
    default sorted policy only for a predicted gain above the margin
    calibrated on a validation batch at training time.  Whole-batch
    time with those policies against every member on the default (median of
    50 graph replays each)."""
    from paper_1101_0091_gb300 import selector as sel
    cm = sel.CostModel.load(os.path.join(COST_MODEL_DIR, "batch.bin"))
    X = np.array([spmv.features(A, 4) for A in As])
    choice, _ = cm.select_guarded(X, sel.BATCH_DEFAULT)
    margin = cm.margin
    cm.close()
    names = [p[0] for p in sel.BATCH_POLICIES]
    batch.set_policies([sel.BATCH_POLICIES[c][1] for c in choice])
    t_sel = statistics.median(timer.run(lambda: batch.apply(stream), 50, 5)["per_ms"]) / 1e3
    batch.set_policies([sel.BATCH_POLICIES[sel.BATCH_DEFAULT][1]] * len(As))
    t_def = statistics.median(timer.run(lambda: batch.apply(stream), 50, 5)["per_ms"]) / 1e3
    return {"model": "paper_1101_0091_gb300/cost_models/batch.bin",
            "margin": None if margin is None or margin == float("inf") else margin,
            "margin_kind": "calibrated on a validation batch (null: keep the default)" if margin is not None
            else "uncalibrated default",
            "choices": {names[v]: int((choice == v).sum()) for v in range(len(names))},
            "gflops_learned": round(flops / t_sel / 1e9, 1), "gflops_default_sorted": round(flops / t_def / 1e9, 1),
            "learned_over_default": round(t_def / t_sel, 4)}


def batch_selector(args, As, batch, timer, stream, flops, spmv):
    """Cost model for batch members: trained on generated members, evaluated on
    every n-th member against the exhaustive sweep of all row policies, then
    used to pick every member's policy in the full batched launch."""
    import tempfile
    from paper_1101_0091_gb300 import selector as sel
    t0 = time.time()
    ctx = sel.BatchContext(sel.batch_background(), stream)
    train = sel.build_dataset(sel.batch_training_matrices(args.selector_train), "batch", stream, batch_ctx=ctx)
    cm = sel.train_model(train, len(sel.BATCH_POLICIES), epochs=sel.BATCH_EPOCHS)
    cal = sel.calibrate_margin(cm, sel.validation_members(), stream)
    ckpt = os.path.join(tempfile.gettempdir(), "spmv_batch_cost_model.bin")
    cm.save(ckpt)
    t_train = time.time() - t0
    idx = list(range(0, len(As), args.selector_stride))
    ev = sel.build_dataset([As[i] for i in idx], "batch", stream, batch_ctx=ctx)
    ctx.close()
    choice, _ = cm.select_guarded(ev.X, sel.BATCH_DEFAULT)
    names = [p[0] for p in sel.BATCH_POLICIES]
    best_fixed = int(ev.times.sum(axis=0).argmin())
    Xall = np.array([spmv.features(A, 4) for A in As])
    ch_all, _ = cm.select_guarded(Xall, sel.BATCH_DEFAULT)
    batch.set_policies([sel.BATCH_POLICIES[c][1] for c in ch_all])
    t_sel = statistics.median(timer.run(lambda: batch.apply(stream), 50, 5)["per_ms"]) / 1e3
    batch.set_policies([sel.BATCH_POLICIES[sel.BATCH_DEFAULT][1]] * len(As))
    t_def = statistics.median(timer.run(lambda: batch.apply(stream), 50, 5)["per_ms"]) / 1e3
    return {"training_members": args.selector_train, "train_and_sweep_s": round(t_train, 1),
            "guard_calibration": cal,
            "evaluated_members": len(idx), "regret_learned": sel.regret(ev.times, choice),
            "regret_default_" + names[sel.BATCH_DEFAULT]: sel.fixed_choice_regret(ev.times, sel.BATCH_DEFAULT),
            "regret_best_fixed_" + names[best_fixed]: sel.fixed_choice_regret(ev.times, best_fixed),
            "choices_all_members": {names[v]: int((ch_all == v).sum()) for v in range(len(names))},
            "batch_gflops_learned_policies": round(flops / t_sel / 1e9, 1),
            "batch_gflops_default_policy": round(flops / t_def / 1e9, 1)}


SELECTOR_KS = (1, 4, 16)   # right-hand-side counts of the plan selector's training samples


def plan_selector(args, A, timer, stream, tr, spmv):
    """Cost model for single products: trained on generated matrices, picks the
    kernel for this workload; its time against the default kernel and the sweep."""
    import torch
    from paper_1101_0091_gb300 import selector as sel
    t0 = time.time()
    train = sel.build_dataset(sel.training_matrices(args.selector_train, seed=1000, scale=0.25), "plan", stream,
                              ks=SELECTOR_KS)
    cm = sel.train_model(train, len(sel.PLAN_VARIANTS))
    t_train = time.time() - t0
    sweep = sel.sweep_plan(A, stream, k=args.k)
    choice, _ = cm.select(spmv.features(A, args.k))
    c = int(choice[0])
    names = [v[0] for v in sel.PLAN_VARIANTS]
    return {"training_matrices": args.selector_train, "training_k": list(SELECTOR_KS), "k": args.k,
            "train_and_sweep_s": round(t_train, 1), "chosen": names[c], "best_in_sweep": names[int(sweep.argmin())],
            "gflops_chosen": round(tr.flops / sweep[c] / 1e9, 1),
            "gflops_default_" + names[sel.PLAN_DEFAULT]: round(tr.flops / sweep[sel.PLAN_DEFAULT] / 1e9, 1),
            "gflops_best": round(tr.flops / sweep.min() / 1e9, 1),
            "regret": round(float(sweep[c] / sweep.min() - 1), 4)}


CONFIG_SECTIONS = ("laplace2d_256", "eigen_6201600", "powerlaw_batch512")
_SECTION_ALIASES = {"laplace": "laplace2d_256", "eigen": "eigen_6201600", "batch": "powerlaw_batch512"}
_TOP_ONLY = ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data", "paper_context", "machine")


def config_sections(args) -> list:
    """The configurations measured beside the headline in one run."""
    c = args.configs
    if c == "auto":
        default = (args.workload == "poisson3d_280" and args.k == 1 and args.variant == "crs_l1"
                   and not args.fp32_val and not args.no_forms)
        return list(CONFIG_SECTIONS) if default else []
    if c == "none":
        return []
    if c == "all":
        return list(CONFIG_SECTIONS)
    return [_SECTION_ALIASES.get(x, x) for x in c.split(",") if x]


def run_config(name, args, torch, spmv, pm, timer, stream, world, rank) -> dict:
    """One configuration section of the default line, bounded in time: the 2D
    Laplacian with k columns and both value storages (first and fourth
    configurations), the eigenproblem-shaped matrix (third), and the uneven
    batch (fifth; its own timed persistent launches, forms and cost model)."""
    import types
    if name == "laplace2d_256":
        return laplace_section(torch, spmv, pm, stream, with_cpu=rank == 0 and not args.no_cpu)
    if name == "eigen_6201600":
        return eigen_section(torch, spmv, pm, timer, stream, steps=50, with_cpu=rank == 0 and not args.no_cpu)
    if name == "powerlaw_batch512":
        sub = types.SimpleNamespace(**vars(args))
        sub.workload, sub.steps, sub.warmup, sub.no_forms, sub.selector = "powerlaw_batch512", 50, 5, False, False
        sec = batch_workload(sub, torch, spmv, pm, timer, stream, world, rank)
        for k in _TOP_ONLY:
            sec.pop(k, None)
        return sec
    raise ValueError(name)


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    import paper_1101_0091_gb300 as spmv
    from paper_1101_0091_gb300 import perfmodel as pm

    rank, world, local = dist_info()
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    spmv.load()
    stream = torch.cuda.Stream()
    timer = Timer(torch, stream, world, local)
    machine = None if args.no_probes else probe_machine(spmv)
    if args.workload.startswith("powerlaw_batch"):
        line = batch_workload(args, torch, spmv, pm, timer, stream, world, rank)
    else:
        line = single_workload(args, torch, spmv, pm, timer, stream, world, rank)
    if machine:
        line["machine"] = machine
    configs = config_sections(args)
    if configs:
        line["configs"] = {}
        for name in configs:
            t0 = time.perf_counter()
            try:
                sec = run_config(name, args, torch, spmv, pm, timer, stream, world, rank)
            except Exception as e:  # the headline stays; the failed section says why
                sec = {"error": f"{type(e).__name__}: {e}"}
            sec["section_wall_s"] = round(time.perf_counter() - t0, 1)
            line["configs"][name] = sec
            torch.cuda.synchronize()
    for fn in LATE_HOST_WORK:
        fn()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
