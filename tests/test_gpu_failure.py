"""Failure detection without a GPU fault: the device-side bounded wait gives up
and reports a status (context stays usable), and the host-side deadline wait
returns a timeout while work is still running."""
import numpy as np
import pytest

import gen
from gpu_util import assert_close, run

pytestmark = pytest.mark.gpu


def test_device_wait_times_out_and_context_survives(lib):
    with pytest.raises(lib.SpmvError) as e:
        lib.spmv_selftest_wait_timeout(20_000)   # 20 ms on a phase that nothing completes
    assert e.value.status == 5  # SPMV_ERR_TIMEOUT
    # the context is intact: a product still runs and is correct
    A = gen.poisson3d_var(20)
    B = gen.uniform(A.n_cols, seed=3)
    with lib.Plan.from_csr(A, variant=lib.SPMV_CRS_STAGED) as p:
        assert_close(run(p, B), A, B)
    with pytest.raises(lib.SpmvError) as e:
        lib.spmv_selftest_wait_timeout(0)
    assert e.value.status == 1


def test_host_deadline_wait(lib):
    import torch
    if not hasattr(torch.cuda, "_sleep"):
        pytest.skip("no spin kernel in this torch")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        torch.cuda._sleep(int(1.5e9))            # ~0.7 s of spinning at 2 GHz, bounded
    with pytest.raises(lib.SpmvError) as e:
        lib.spmv_wait(s.cuda_stream, 5)
    assert e.value.status == 5
    lib.spmv_wait(s.cuda_stream, 20_000)
    lib.spmv_wait(s.cuda_stream, 0)              # finished work: immediate success
    with pytest.raises(lib.SpmvError):
        lib.spmv_wait(s.cuda_stream, -1)
