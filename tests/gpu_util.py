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


def assert_close(y, A, B, tol=TOL_FP64, f32val=False, exact=False):
    ref = oracle.spmm(A, B, f32val=f32val) if B.ndim == 2 else (
        oracle.spmm(A, B.reshape(-1, 1), f32val=f32val)[:, 0] if f32val else oracle.spmv(A, B))
    if exact:
        assert np.array_equal(y, ref), "not bit-exact"
        return 0.0
    r = oracle.max_err_ratio(y, ref, oracle.abs_scale(A, B), tol)
    assert r <= 1.0, f"max error ratio {r}"
    return r
