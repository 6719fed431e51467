#!/usr/bin/env python3
"""Benchmark of the CRS spMVM C = A*B on GB300.

Workload (default): the 3D 7-point variable-coefficient Poisson stencil on a
280^3 grid (N = 21,952,000 rows, 153,193,600 nonzeros, FP64 CRS), the stand-in
for the paper's sAMG matrix.  One step = one product C = A*B with the plan's
default kernel (CRS_L1: thread per row, val/col slices of the CTA 152 positions
ahead prefetched into L2 by the TMA engine).  Inputs (2.28 GB) exceed L2
(129 MB), so no flush is needed between steps.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle instead.
Under torchrun each rank runs an independent replica (the path does not shard
over GPUs here) and `value` is the sum over ranks.
"""
from __future__ import annotations

import argparse
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
    "poisson3d_280": "3D 7-point variable-coefficient Poisson stencil, 280^3 grid, N=21,952,000, nnz=153,193,600, FP64 CRS, B~U[-1,1) seed 0",
    "poisson3d_160": "3D 7-point variable-coefficient Poisson stencil, 160^3 grid, N=4,096,000, nnz=28,518,400, FP64 CRS (profiling size)",
    "eigen_6201600": "symmetric eigenproblem-shaped matrix, N=6,201,600 (400 x 15,504), ~13.8 nnz/row, FP64 CRS",
}
VARIANTS = {"crs_staged": (1, 1), "crs_l1": (2, 1), "crs_l2": (3, 1), "crs_l4": (4, 1), "crs_l8": (5, 1),
            "crs_l16": (6, 1), "crs_l32": (7, 1), "sell_s1": (8, 1), "sell_s256": (8, 256), "sell_s4096": (8, 4096)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="poisson3d_280", choices=sorted(WORKLOADS))
    ap.add_argument("--variant", default="crs_l1", choices=sorted(VARIANTS))
    ap.add_argument("--fp32-val", action="store_true", help="store val in FP32 (FP64 accumulation)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer measurement")
    return ap.parse_args()


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def load_workload(name):
    import gen
    if name.startswith("poisson3d_"):
        A = gen.poisson3d_var(int(name.split("_")[1]), seed=0)
    elif name == "eigen_6201600":
        A = gen.eigen_shaped(6_201_600, seed=0)
    else:
        raise ValueError(name)
    return A, gen.uniform(A.n_cols, seed=0)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_fingerprint() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_1101_0091_gb300", "csrc"))):
        with open(os.path.join(ROOT, "paper_1101_0091_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(f"{kernel}/{workload}")
    if not e or e.get("source_fingerprint") != kernel_fingerprint():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def time_oracle(A, B, steps: int, budget_s: float = 20.0):
    """Time the oracle's plain FP64 loop (single thread) on the full product,
    at most `steps` runs or `budget_s` seconds."""
    import oracle
    oracle.spmv(A, B)  # load / warm
    ts = []
    t_end = time.perf_counter() + budget_s
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        oracle.spmv(A, B)
        ts.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end:
            break
    return ts


def reference_arm(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    A, B = load_workload(args.workload)
    flops = 2 * A.nnz
    ts = time_oracle(A, B, args.steps + args.warmup, budget_s=120.0)
    ts = ts[min(args.warmup, len(ts) - 1):] if len(ts) > 1 else ts
    t = sum(ts) / len(ts)
    value = flops / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GFlop/s", "n_gpus": args.gpus,
            "steps": len(ts), "warmup": args.warmup, "ms_per_step": round(t * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": WORKLOADS[args.workload]},
            "cpu_baseline": {"value": round(value, 4), "unit": "GFlop/s", "cores": 1, "kind": "oracle",
                             "sample": f"full product, {len(ts)} timed runs of the single-threaded FP64 CRS loop"},
            "e2e": {"value": round(value, 4), "unit": "GFlop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    import paper_1101_0091_gb300 as spmv
    from paper_1101_0091_gb300 import perfmodel as pm

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    spmv.load()
    A, Bh = load_workload(args.workload)
    vid, sigma = VARIANTS[args.variant]
    plan = spmv.Plan.from_csr(A, variant=vid, sell_sigma=sigma, val_fp32=args.fp32_val)
    stream = torch.cuda.Stream()
    B = torch.from_numpy(Bh).cuda()
    C = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
    traffic = pm.gpu_min_traffic(A.n_rows, A.n_cols, A.nnz, val_bytes=4 if args.fp32_val else 8)
    hbm_peak, peak_kind = measured_peaks()

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    stream.wait_stream(torch.cuda.current_stream())
    for _ in range(args.warmup):
        plan.apply(B, C, stream)
    plan.check(stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        ev[0].record(stream)
        for i in range(args.steps):
            plan.apply(B, C, stream)
            ev[i + 1].record(stream)
        stream.synchronize()
        wall = time.perf_counter() - t0
    barrier()
    plan.check(stream)
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    t_step = total_ms / 1e3 / args.steps
    flops_all = traffic.flops * world
    value = flops_all / t_step / 1e9
    kern_s = statistics.mean(per) / 1e3
    achieved = traffic.bytes_min / kern_s / 1e9

    # end to end through the C ABI from pinned host buffers (H2D of B, D2H of C inside the timed region)
    e2e = None
    if not args.no_e2e:
        Bpin = torch.from_numpy(Bh).pin_memory()
        Cpin = torch.empty(A.n_rows, dtype=torch.float64).pin_memory()
        for _ in range(2):
            plan.apply_host_ptr(Bpin.data_ptr(), 1, Cpin.data_ptr(), stream)
        e2e_steps = max(3, min(args.steps, 20))
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            plan.apply_host_ptr(Bpin.data_ptr(), 1, Cpin.data_ptr(), stream)
        e2e_t = (time.perf_counter() - t0) / e2e_steps
        if world > 1:
            t = torch.tensor([e2e_t], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            e2e_t = float(t.item())
        e2e = {"value": round(flops_all / e2e_t / 1e9, 3), "unit": "GFlop/s", "h2d_bytes_per_step": 8 * A.n_cols,
               "d2h_bytes_per_step": 8 * A.n_rows}

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GFlop/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_step * 1e3, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload], "kernel": args.variant,
                   "val_storage": "f32" if args.fp32_val else "f64", "n_rows": A.n_rows, "nnz": A.nnz,
                   "l2": f"inputs larger than L2 ({traffic.bytes_min / 1e9:.2f} GB vs 129 MB), no flush",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "hbm_gbs": round(achieved, 1),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                     "frac": round(achieved / hbm_peak, 4), "peak_kind": peak_kind,
                     "traffic": ncu_traffic(args.variant, args.workload),
                     "algorithmic_bytes_per_launch": traffic.bytes_min},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "wall_s_timed": round(wall, 4),
    }
    if rank == 0 and not args.no_cpu:
        ts = time_oracle(A, Bh, 3)
        tc = min(ts)
        line["cpu_baseline"] = {"value": round(traffic.flops / tc / 1e9, 4), "unit": "GFlop/s", "cores": 1,
                                "kind": "oracle", "sample": f"full product, best of {len(ts)} single-threaded runs"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
