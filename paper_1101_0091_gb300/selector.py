"""Learned variant selection: exhaustive timed sweeps of this library's own
kernels, the MLP cost model trained on them (forward, backward and Adam run in
the library's CUDA kernels), and the regret of its choices.

Two contexts share the code:
* "plan":  single-matrix products of k columns (k is a feature; one sample
           per matrix and k); the variants are the plan kernels
           (CRS_L1/L2/L4/L8/L32, CRS_STAGED, SELL-32 with sigma 1/256/4096).
* "batch": members of a batched launch, k = 4; the variants are the batch row
           policies (fixed 1/2/4/8/32 lanes per row, adaptive, sorted).

Targets are log(seconds); the network predicts one value per variant and the
selection is the argmin.  Training matrices come from seeds >= 1000 of the
input generators (the evaluation workloads use seed 0).
"""
from __future__ import annotations

import math
import statistics
from dataclasses import dataclass, field

import numpy as np

from . import Batch, Plan, features
from . import _binding_model as bm

PLAN_VARIANTS = [("crs_l1", 2, 1), ("crs_l2", 3, 1), ("crs_l4", 4, 1), ("crs_l8", 5, 1), ("crs_l32", 7, 1),
                 ("crs_staged", 1, 1), ("sell_s1", 8, 1), ("sell_s256", 8, 256), ("sell_s4096", 8, 4096)]
PLAN_DEFAULT = 0          # CRS_L1, the plan's AUTO kernel
BATCH_POLICIES = [("l1", 0), ("l2", 1), ("l4", 2), ("l8", 3), ("l32", 4), ("adapt", 5), ("sorted", 6)]
BATCH_DEFAULT = 6         # sorted, the batch's default policy
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


def sweep_batch(A, stream, k: int = 4, reps: int = 5, target_nnz: int = 2_000_000) -> np.ndarray:
    """Seconds per member copy for every batch policy: the member is replicated
    R times in one batched launch (R copies reach ~target_nnz nonzeros), so the
    launch overhead is amortised as it is inside a real batch."""
    torch = _torch()
    R = max(1, min(512, math.ceil(target_nnz / max(A.nnz, 1))))
    B = torch.from_numpy(np.ones((A.n_cols, k))).cuda()
    Cs = [torch.empty((A.n_rows, k), dtype=torch.float64, device="cuda") for _ in range(R)]
    stream.wait_stream(torch.cuda.current_stream())
    out = np.zeros(len(BATCH_POLICIES))
    with Plan.from_csr(A) as p:
        with Batch([p] * R, k) as b:
            b.set_io([B] * R, Cs)
            for i, (_, pol) in enumerate(BATCH_POLICIES):
                b.set_policies([pol] * R)
                out[i] = event_time(lambda: b.apply(stream), stream, reps) / R
    return out


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


def build_dataset(mats, context: str, stream, k: int = None, ks=None) -> Dataset:
    """One sample per matrix and k (ks, default [k]; k defaults to 1 for the
    plan context and 4 for the batch context)."""
    k = (1 if context == "plan" else 4) if k is None else k
    ks = [k] if ks is None else list(ks)
    X, TT = [], []
    for A in mats:
        for kk in ks:
            X.append(features(A, kk))
            TT.append(sweep_plan(A, stream, k=kk) if context == "plan" else sweep_batch(A, stream, kk))
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
        if handle is not None:
            self.handle = handle
        else:
            self.handle = bm.spmv_model_create(N_FEATURES, hidden, n_variants,
                                               init_params(N_FEATURES, hidden, n_variants, seed))

    @classmethod
    def load(cls, path: str) -> "CostModel":
        return cls(0, handle=bm.spmv_model_load(path))

    def save(self, path: str) -> None:
        bm.spmv_model_save(self.handle, path)

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
