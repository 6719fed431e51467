"""Pins of the oracle's feature vector on matrices whose features are known by hand."""
import numpy as np
import pytest

import gen
from oracle import features as F


def test_identity_features():
    n = 8
    I = gen.CSR(n, n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n))
    f = F.features(I, k=4)
    expect = np.zeros(F.N_FEATURES)
    expect[1] = 1.0            # every row has length 1 -> bin 1
    expect[F.N_BINS + 1] = 1.0
    expect[26] = np.log2(9)
    expect[27] = np.log2(9)
    expect[28] = 1.0
    expect[29] = 1.0
    expect[33] = 2.0
    assert np.array_equal(f, expect)


def test_laplace_4x4_features():
    """4x4 grid: 4 corner rows of length 3, 8 edge rows of 4, 4 inner rows of 5."""
    A = gen.laplace2d(4)
    f = F.features(A)
    assert f[2] == 4 / 16                 # length 3 -> bin 2 ([2, 4))
    assert f[3] == 12 / 16                # lengths 4, 5 -> bin 3 ([4, 8))
    assert f[F.N_BINS + 2] == 12 / 64
    assert f[F.N_BINS + 3] == 52 / 64
    assert f[28] == 64 / 16
    assert f[29] == np.log2(6)
    mean = 4.0
    std = np.sqrt((4 * 1 + 8 * 0 + 4 * 1) / 16)
    assert f[30] == pytest.approx(std / (1 + mean), rel=1e-15)
    assert f[31] == 4 / 16                # the +-nx neighbours
    # column spans by hand: grid rows y=0 and y=3 give 4+5+5+5 each, y=1 and y=2 give 8 per row
    assert f[32] == (19 + 32 + 32 + 19) / (16 * 16)
    assert f[33] == 0.0


def test_bins():
    L = np.array([0, 1, 2, 3, 4, 7, 8, 2047, 2048, 100000])
    assert F.length_bin(L).tolist() == [0, 1, 2, 2, 3, 3, 4, 11, 12, 12]
