"""Helpers of the GPU parity tests: device copies, running a plan, and the
tolerance check against the oracle (|y - y_ref| <= tol * sum_j |a_ij b_j| per
row and right-hand side)."""
import numpy as np

import oracle

TOL_FP64 = 1e-13
TOL_FP32VAL = 2e-7


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def run(plan, B: np.ndarray, k: int | None = None, fill=np.nan):
    """Apply a plan to host B (1-D or n_cols x k) and return C on the host."""
    import torch
    Bd = dev(B)
    if B.ndim == 1:
        C = torch.full((plan.n_rows,), fill, dtype=torch.float64, device="cuda")
        plan.apply(Bd, C)
    else:
        C = torch.full((plan.n_rows, B.shape[1]), fill, dtype=torch.float64, device="cuda")
        plan.apply_block(Bd, C, k)
    plan.check()
    return host(C)


def attribution(y, ref, A, B, tol, f32val=False) -> str:
    """For the worst entry of a failed check: the distances of the kernel's and
    the oracle's results from a compensated (Dot2) evaluation of the same row,
    which tells which side carries the error."""
    import gen
    if f32val:
        A = gen.CSR(A.n_rows, A.n_cols, A.row_ptr, A.col_idx, A.val.astype(np.float32).astype(np.float64))
    ex = oracle.spmm_dot2(A, B)
    scale = oracle.abs_scale(A, B)
    ratio = np.abs(y - ref) / np.maximum(tol * scale, np.finfo(np.float64).tiny)
    i = np.unravel_index(int(np.nanargmax(np.where(np.isnan(y), np.inf, ratio))), ratio.shape)
    return (f"worst entry {tuple(int(x) for x in i)}: |y - oracle| = {abs(y[i] - ref[i]):.3e}, "
            f"|y - dot2| = {abs(y[i] - ex[i]):.3e}, |oracle - dot2| = {abs(ref[i] - ex[i]):.3e}, "
            f"tol * sum|ab| = {tol * scale[i]:.3e}")


def assert_close(y, A, B, tol=TOL_FP64, f32val=False, exact=False):
    ref = oracle.spmm(A, B, f32val=f32val) if B.ndim == 2 else (
        oracle.spmm(A, B.reshape(-1, 1), f32val=f32val)[:, 0] if f32val else oracle.spmv(A, B))
    if exact:
        assert np.array_equal(y, ref), "not bit-exact"
        return 0.0
    r = oracle.max_err_ratio(y, ref, oracle.abs_scale(A, B), tol)
    assert r <= 1.0, f"max error ratio {r}; " + attribution(y, ref, A, B, tol, f32val)
    return r
