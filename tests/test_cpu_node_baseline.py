"""The OpenMP CPU node baseline (timed by bench.py beside the GPU kernels)
computes the oracle's result bit for bit: same loop, same order per row."""
import numpy as np
import pytest

import gen
import oracle

baselines = pytest.importorskip("baselines")


@pytest.mark.parametrize("name", ["laplace", "poisson", "powerlaw"])
def test_openmp_loop_equals_oracle(name):
    if not baselines.available():
        pytest.skip("OpenMP not available to gcc here")
    A = {"laplace": lambda: gen.laplace2d(64), "poisson": lambda: gen.poisson3d_var(20),
         "powerlaw": lambda: gen.powerlaw(20_000, seed=4)}[name]()
    B = gen.uniform(A.n_cols, seed=1)
    assert np.array_equal(baselines.spmv(A, B), oracle.spmv(A, B))
