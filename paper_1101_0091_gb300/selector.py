"""Learned variant selection: exhaustive timed sweeps of this library's own
kernels, the MLP cost model trained on them (forward, backward and Adam run in
the library's CUDA kernels), and the regret of its choices.

Two contexts share the code:
* "plan":  single-matrix products of k columns (k is a feature; one sample
           per matrix and k); the variants are the plan kernels
           (CRS_L1/L2/L4/L8/L32, CRS_STAGED, SELL-32 with sigma 1/256/4096).
* "batch": members of a batched launch, k = 4; the variants are the batch row
           policies (fixed 1/2/4/8/32 lanes per row, adaptive, sorted), each
           member timed inside a mixed batch of other members; selection is
           guarded: a member leaves the default (sorted) policy only for a
           predicted gain above a margin calibrated on a validation batch.

Targets are log(seconds); the network predicts one value per variant and the
selection is the argmin.  Training matrices come from seeds >= 1000 of the
input generators (the evaluation workloads use seed 0).
"""
from __future__ import annotations

import json
import math
import os
import statistics
from dataclasses import dataclass, field

import numpy as np

from . import Batch, Plan, features
from . import _binding_model as bm

PLAN_VARIANTS = [("crs_l1", 2, 1), ("crs_l2", 3, 1), ("crs_l4", 4, 1), ("crs_l8", 5, 1), ("crs_l32", 7, 1),
                 ("crs_staged", 1, 1), ("sell_s1", 8, 1), ("sell_s256", 8, 256), ("sell_s4096", 8, 4096)]
PLAN_DEFAULT = 0          # CRS_L1, plain CRS (AUTO runs it on all but scattered matrices)
BATCH_POLICIES = [("l1", 0), ("l2", 1), ("l4", 2), ("l8", 3), ("l32", 4), ("adapt", 5), ("sorted", 6)]
BATCH_DEFAULT = 6         # sorted, the batch's default policy
BATCH_MARGIN = 0.25       # guard margin of an uncalibrated batch model (a predicted gain above ~28 %)
BATCH_MARGINS = (0.05, 0.1, 0.25, 0.5)   # candidates of the calibration, smallest first
BATCH_EPOCHS = 800        # fewer steps than the plan model: the batch targets differ little and are noisy
N_FEATURES = 34


def _torch():
    import torch
    return torch


def event_time(fn, stream, reps: int = 7, warm: int = 2) -> float:
    """Median seconds of `fn` over `reps` launches (CUDA events on `stream`)."""
    torch = _torch()
    for _ in range(warm):
        fn()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record(stream)
    for i in range(reps):
        fn()
        ev[i + 1].record(stream)
    stream.synchronize()
    return statistics.median(ev[i].elapsed_time(ev[i + 1]) for i in range(reps)) / 1e3


# ------------------------------------------------------------------- sweeps

def sweep_plan(A, stream, reps: int = 7, k: int = 1) -> np.ndarray:
    """Seconds of one product of k columns with every plan variant."""
    torch = _torch()
    shape_b = (max(A.n_cols, 1),) if k == 1 else (max(A.n_cols, 1), k)
    B = torch.ones(shape_b, dtype=torch.float64, device="cuda")
    C = torch.empty((max(A.n_rows, 1),) if k == 1 else (max(A.n_rows, 1), k), dtype=torch.float64, device="cuda")
    stream.wait_stream(torch.cuda.current_stream())
    out = np.zeros(len(PLAN_VARIANTS))
    with Plan.from_csr(A) as p:
        fn = (lambda: p.apply(B, C, stream)) if k == 1 else (lambda: p.apply_block(B, C, k, stream))
        for i, (_, vid, sigma) in enumerate(PLAN_VARIANTS):
            p.set_variant(vid, sigma)
            out[i] = event_time(fn, stream, reps)
    return out


def batch_background(count: int = 48, seed: int = 5000):
    """The mixed batch that training members are timed inside: members of the
    uneven-batch generator with seeds of their own (>= 5000)."""
    import gen
    return [gen.powerlaw_batch_member(i, seed=seed) for i in range(count)]


class BatchContext:
    """Times a member's row policies inside a mixed batch: the member (one
    copy or a few; `copies` > 1, or None for as many copies as the
    background has nonzeros), each copy a plan of its own with its own B and
    C so that it streams its arrays from HBM as a member of a real batch
    does, placed in the middle of a background of other members on the
    default (sorted) policy.  The target of a policy is the time of that whole
    batch: only the differences between a member's policies matter to the
    selection, and a difference of whole-batch times is what the selection
    changes.  Why this form, as measured on GB300: a member's cost is not
    additive.  A policy whose work items are long chains of dependent gathers
    (one-entry rows on one lane each, 32 passes per item) leaves one warp
    busy for tens of microseconds, and where such an item starts late it
    stretches the whole batch; one such member added 20 us to a 115 us batch
    while its own work was 4 % of it.  Many copies of the member spread those
    items over the batch and hide that tail, and copies that share one set of
    arrays find them in L2; both made the adaptive policy look faster than it
    is."""

    def __init__(self, background, stream, k: int = 4, reps: int = 9, copies: int | None = 4,
                 max_copies: int = 128):
        torch = _torch()
        self.stream, self.k, self.reps, self.max_copies, self.copies = stream, k, reps, max_copies, copies
        self.bg = background
        self.bg_plans = [Plan.from_csr(A) for A in background]
        self.bg_B = [torch.from_numpy(np.ones((A.n_cols, k))).cuda() for A in background]
        self.bg_C = [torch.empty((A.n_rows, k), dtype=torch.float64, device="cuda") for A in background]
        self.bg_nnz = sum(A.nnz for A in background)
        stream.wait_stream(torch.cuda.current_stream())

    def sweep(self, A) -> np.ndarray:
        torch = _torch()
        k, stream = self.k, self.stream
        R = self.copies or max(1, min(self.max_copies, math.ceil(self.bg_nnz / max(A.nnz, 1))))
        copies = [Plan.from_csr(A) for _ in range(R)]
        Bc = [torch.from_numpy(np.ones((A.n_cols, k))).cuda() for _ in range(R)]
        Cc = [torch.empty((A.n_rows, k), dtype=torch.float64, device="cuda") for _ in range(R)]
        stream.wait_stream(torch.cuda.current_stream())
        out = np.zeros(len(BATCH_POLICIES))
        try:
            # member order: the copies spread evenly through the background (one copy: in its middle)
            nb = len(self.bg_plans)
            slots = sorted(((q + 0.5) * nb / R, "m", q) for q in range(R))
            order, q = [], 0
            for i in range(nb):
                while q < R and slots[q][0] <= i:
                    order.append(("m", slots[q][2]))
                    q += 1
                order.append(("bg", i))
            order += [("m", slots[x][2]) for x in range(q, R)]
            plans = [self.bg_plans[x] if t == "bg" else copies[x] for t, x in order]
            Bs = [self.bg_B[x] if t == "bg" else Bc[x] for t, x in order]
            Cl = [self.bg_C[x] if t == "bg" else Cc[x] for t, x in order]
            with Batch(plans, k) as b:
                b.set_io(Bs, Cl)
                for v, (_, pol) in enumerate(BATCH_POLICIES):
                    b.set_policies([BATCH_POLICIES[BATCH_DEFAULT][1] if t == "bg" else pol for t, _ in order])
                    out[v] = event_time(lambda: b.apply(stream), stream, self.reps)
        finally:
            for p in copies:
                p.close()
        return out

    def close(self):
        for p in self.bg_plans:
            p.close()
        self.bg_plans = []


# ------------------------------------------------------------- training set

def training_matrices(count: int, seed: int = 1000, scale: float = 1.0):
    """Generated matrices of several families (seeds >= 1000): 3D and 2D
    stencils, eigenproblem-shaped, power-law rows, constant-length rows."""
    import gen
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        fam = i % 5
        s = seed + i
        if fam == 0:
            out.append(gen.poisson3d_var(int(rng.integers(16, int(16 + 80 * scale) + 1)), seed=s))
        elif fam == 1:
            out.append(gen.laplace2d(int(rng.integers(48, int(48 + 900 * scale) + 1))))
        elif fam == 2:
            n = int(rng.integers(20_000, int(20_000 + 1_500_000 * scale) + 1))
            out.append(gen.eigen_shaped(n, seed=s, window=int(2 ** rng.integers(8, 21)),
                                        pairs=int(rng.integers(1, 9)), band_p=float(rng.uniform(0.2, 1.0))))
        elif fam == 3:
            n = int(rng.integers(5_000, int(5_000 + 400_000 * scale) + 1))
            out.append(gen.powerlaw(n, alpha=float(rng.uniform(1.6, 3.2)), lmax=int(rng.choice([16, 128, 2000])),
                                    seed=s))
        else:
            L = int(rng.choice([1, 2, 3, 5, 8, 13, 24, 48, 96, 200]))
            n = int(rng.integers(5_000, int(5_000 + 200_000 * scale) + 1))
            out.append(gen.powerlaw(n, lmin=L, lmax=L, seed=s))
    return out


@dataclass
class Dataset:
    X: np.ndarray            # features, M x 34 (float64)
    T: np.ndarray            # log seconds, M x V
    times: np.ndarray        # seconds, M x V
    names: list = field(default_factory=list)


def build_dataset(mats, context: str, stream, k: int = None, ks=None, batch_ctx: "BatchContext" = None) -> Dataset:
    """One sample per matrix and k (ks, default [k]; k defaults to 1 for the
    plan context and 4 for the batch context).  In the batch context the
    members are timed inside batch_ctx's mixed batch (a default one when none
    is given)."""
    k = (1 if context == "plan" else 4) if k is None else k
    ks = [k] if ks is None else list(ks)
    own_ctx = context != "plan" and batch_ctx is None
    if own_ctx:
        batch_ctx = BatchContext(batch_background(), stream, k=k)
    X, TT = [], []
    for A in mats:
        for kk in ks:
            X.append(features(A, kk))
            TT.append(sweep_plan(A, stream, k=kk) if context == "plan" else batch_ctx.sweep(A))
    if own_ctx:
        batch_ctx.close()
    times = np.array(TT)
    return Dataset(np.array(X), np.log(times), times)


# -------------------------------------------------------------------- model

def init_params(F: int, H: int, V: int, seed: int) -> np.ndarray:
    """He-uniform weights, zero biases (the random draw is an input of the model)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((F, H), (H, H), (H, V)):
        lim = math.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, (fan_out, fan_in)).ravel())
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


class CostModel:
    """Owns a spmv_model_handle; training and selection run in the library."""

    def __init__(self, n_variants: int, hidden: int = 64, seed: int = 0, handle=None):
        self.margin = None          # calibrated guard margin (None: not calibrated; inf: keep the default)
        if handle is not None:
            self.handle = handle
        else:
            self.handle = bm.spmv_model_create(N_FEATURES, hidden, n_variants,
                                               init_params(N_FEATURES, hidden, n_variants, seed))

    @classmethod
    def load(cls, path: str) -> "CostModel":
        cm = cls(0, handle=bm.spmv_model_load(path))
        side = path + ".json"
        if os.path.exists(side):
            with open(side) as f:
                m = json.load(f).get("margin")
            cm.margin = math.inf if m is None else float(m)
        return cm

    def save(self, path: str) -> None:
        bm.spmv_model_save(self.handle, path)
        if self.margin is not None:
            with open(path + ".json", "w") as f:
                json.dump({"margin": None if math.isinf(self.margin) else self.margin,
                           "about": "guard margin calibrated on a validation batch (null: keep the default)"}, f)

    def fit(self, data: Dataset, epochs: int = 2000, lr: float = 3e-3, stream=None) -> list:
        """Full-batch Adam on the masked MSE of log times; returns the loss curve."""
        torch = _torch()
        mean = data.X.mean(axis=0)
        std = data.X.std(axis=0)
        inv = np.where(std > 1e-12, 1.0 / np.where(std > 1e-12, std, 1.0), 0.0)
        bm.spmv_model_set_normalizer(self.handle, mean, inv)
        T = data.T - data.T.mean(axis=1, keepdims=True)  # the argmin needs only differences per matrix
        Xd = torch.from_numpy(data.X.astype(np.float32)).cuda()
        Td = torch.from_numpy(np.nan_to_num(T, nan=0.0).astype(np.float32)).cuda()
        Md = torch.from_numpy(np.isfinite(T).astype(np.float32)).cuda()
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        s = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
        curve = []
        M = data.X.shape[0]
        for e in range(epochs):
            bm.spmv_model_train_step(self.handle, Xd.data_ptr(), Td.data_ptr(), Md.data_ptr(), M, lr,
                                     loss.data_ptr(), s)
            if e % 100 == 0 or e == epochs - 1:
                curve.append(float(loss.item()))
        return curve

    def select(self, X: np.ndarray):
        return bm.spmv_model_select(self.handle, X)

    def select_guarded(self, X: np.ndarray, fallback: int, margin: float | None = None):
        """The network's choice where it predicts a gain above `margin` (default:
        the calibrated margin) over output `fallback`, else `fallback`
        (spmv_model_select_guarded); an infinite margin keeps the fallback."""
        m = self.margin if margin is None else margin
        if m is None:
            m = BATCH_MARGIN
        if math.isinf(m):
            X2 = np.atleast_2d(X)
            return np.full(X2.shape[0], fallback, np.int32), bm.spmv_model_select(self.handle, X2)[1]
        return bm.spmv_model_select_guarded(self.handle, X, fallback, m)

    def close(self):
        if getattr(self, "handle", None) is not None:
            bm.spmv_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_training_matrices(count: int, seed: int = 1000):
    """Generated batch members (seeds >= 1000): members of the uneven-batch
    generator itself (other seeds), power-law rows with varied exponents and
    caps over log-uniform sizes, constant-length rows, stencils."""
    import gen
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        fam = i % 4
        s = seed + i
        n = int(round(math.exp(rng.uniform(math.log(1e3), math.log(2e5)))))
        if fam == 0:
            out.append(gen.powerlaw_batch_member(i, seed=s))
        elif fam == 1:
            out.append(gen.powerlaw(n, alpha=float(rng.uniform(1.6, 3.2)), lmax=int(rng.choice([8, 64, 512, 2000])),
                                    seed=s))
        elif fam == 2:
            L = int(rng.choice([1, 2, 4, 8, 16, 40, 100]))
            out.append(gen.powerlaw(n, lmin=L, lmax=min(L, n), seed=s))
        else:
            out.append(gen.poisson3d_var(int(rng.integers(10, 60)), seed=s))
    return out


def train_model(data: Dataset, n_variants: int, epochs: int = 2000, seed: int = 0) -> CostModel:
    cm = CostModel(n_variants, hidden=64, seed=seed)
    cm.fit(data, epochs=epochs)
    return cm


def batch_time(members, policies, stream, reps: int = 30) -> float:
    """Median seconds of one batched launch of `members` (k = 4) with the given
    row policies (graph replays, CUDA events)."""
    torch = _torch()
    plans = [Plan.from_csr(A) for A in members]
    Bs = [torch.ones((A.n_cols, 4), dtype=torch.float64, device="cuda") for A in members]
    Cs = [torch.empty((A.n_rows, 4), dtype=torch.float64, device="cuda") for A in members]
    stream.wait_stream(torch.cuda.current_stream())
    try:
        with Batch(plans, 4, [int(p) for p in policies]) as b:
            b.set_io(Bs, Cs)
            return event_time(lambda: b.apply(stream), stream, reps=reps, warm=5)
    finally:
        for p in plans:
            p.close()


def calibrate_margin(cm: "CostModel", members, stream, margins=BATCH_MARGINS, tol: float = 0.005) -> dict:
    """Validate the guard against the objective it serves: on a validation
    batch (members of no training or evaluation set), the smallest margin
    whose guarded choices give a whole batch no slower than every member on
    the default policy (within `tol`); infinite (keep the default) if none
    does.  A member's cost inside a batch is not additive (a late work item
    can stretch the whole launch), so the network's per-member predictions are
    not trusted without this check.  Sets cm.margin."""
    X = np.array([features(A, 4) for A in members])
    default = [BATCH_POLICIES[BATCH_DEFAULT][1]] * len(members)
    t_def = batch_time(members, default, stream)
    tried = []
    cm.margin = math.inf
    for m in sorted(margins):
        choice = cm.select_guarded(X, BATCH_DEFAULT, m)[0]
        if np.all(choice == BATCH_DEFAULT):
            cm.margin = m          # from here on the guard keeps every member on the default
            tried.append({"margin": m, "moved": 0, "time_ratio": 1.0})
            break
        t = batch_time(members, [BATCH_POLICIES[c][1] for c in choice], stream)
        tried.append({"margin": m, "moved": int(np.sum(choice != BATCH_DEFAULT)), "time_ratio": round(t / t_def, 4)})
        if t <= (1.0 + tol) * t_def:
            cm.margin = m
            break
    return {"margin": None if math.isinf(cm.margin) else cm.margin, "default_us": round(t_def * 1e6, 1),
            "tried": tried}


def validation_members(count: int = 48, seed: int = 9000):
    """Validation batch of the calibration: uneven-batch members of seeds of their own."""
    import gen
    return [gen.powerlaw_batch_member(i, seed=seed) for i in range(count)]


def regret(times: np.ndarray, choice: np.ndarray) -> dict:
    """Regret of a choice against the exhaustive sweep: sum(t_chosen)/sum(t_best) - 1
    and the mean of the per-matrix ratios minus one."""
    idx = np.arange(times.shape[0])
    t_ch = times[idx, choice]
    t_best = times.min(axis=1)
    return {"total": float(t_ch.sum() / t_best.sum() - 1.0), "mean": float(np.mean(t_ch / t_best) - 1.0),
            "hit_rate": float(np.mean(choice == times.argmin(axis=1)))}


def fixed_choice_regret(times: np.ndarray, v: int) -> dict:
    return regret(times, np.full(times.shape[0], v, dtype=np.int32))


def train_and_save(context: str, count: int, out: str, seed: int = 1000) -> dict:
    """Train a cost model on this GPU and save its checkpoint: the plan model
    on generated matrices at k = 1, 4, 16 (9 kernel variants), or the batch
    model on generated members timed inside a mixed batch (7 row policies)."""
    import time
    torch = _torch()
    stream = torch.cuda.Stream()
    t0 = time.time()
    if context == "plan":
        data = build_dataset(training_matrices(count, seed=seed, scale=0.25), "plan", stream, ks=(1, 4, 16))
        cm = train_model(data, len(PLAN_VARIANTS))
        hit = regret(data.times, cm.select(data.X)[0])
    else:
        ctx = BatchContext(batch_background(), stream)
        data = build_dataset(batch_training_matrices(count, seed=seed), "batch", stream, batch_ctx=ctx)
        ctx.close()
        cm = train_model(data, len(BATCH_POLICIES), epochs=BATCH_EPOCHS)
        cal = calibrate_margin(cm, validation_members(), stream)
        hit = regret(data.times, cm.select_guarded(data.X, BATCH_DEFAULT)[0])
        hit["calibration"] = cal
    cm.save(out)
    cm.close()
    return {"context": context, "samples": int(data.X.shape[0]), "seconds": round(time.time() - t0, 1),
            "training_regret": hit}


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="train a cost model on this GPU and save the checkpoint")
    ap.add_argument("--context", choices=["plan", "batch"], required=True)
    ap.add_argument("--train", type=int, default=100, help="generated training matrices")
    ap.add_argument("--out", required=True)
    ap.add_argument("--seed", type=int, default=1000)
    a = ap.parse_args()
    from . import load
    load()
    print(json.dumps(train_and_save(a.context, a.train, a.out, a.seed)))
