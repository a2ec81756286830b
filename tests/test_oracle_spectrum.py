"""Pins for the oracle's mean subtraction, FFT and whitening."""
import math

import numpy as np

from oracle import spectrum as SP


def _dft(y):
    N = y.shape[0]
    n = np.arange(N)
    k = n[: N // 2]
    W = np.exp(-2j * np.pi * np.outer(k, n) / N)
    return W @ y


def test_half_spectrum_equals_brute_dft():
    rng = np.random.default_rng(1)
    for N in (8, 64, 1024):
        y = rng.standard_normal(N)
        np.testing.assert_allclose(SP.half_spectrum(y), _dft(y), rtol=0, atol=1e-9 * N)


def test_parseval():
    rng = np.random.default_rng(2)
    N = 4096
    y = rng.standard_normal(N)
    A = SP.half_spectrum(y)
    nyq = float(np.sum(y * (-1.0) ** np.arange(N)))
    lhs = float(np.sum(y * y))
    rhs = (abs(A[0]) ** 2 + 2.0 * np.sum(np.abs(A[1:]) ** 2) + nyq ** 2) / N
    assert abs(lhs - rhs) < 1e-9 * lhs


def test_pure_tone_power():
    N, a, k0 = 2048, 0.7, 100
    y = a * np.cos(2 * np.pi * k0 * np.arange(N) / N)
    A = SP.half_spectrum(y)
    assert abs(abs(A[k0]) ** 2 - (N * a / 2) ** 2) < 1e-6 * (N * a / 2) ** 2
    assert np.max(np.abs(np.delete(A, k0))) < 1e-8 * N


def test_real_series_mean_and_padding():
    s = np.array([5, 7, 9, 11, 13], dtype=np.int64)
    y = SP.real_series(s, 8)
    assert y.tolist() == [-4.0, -2.0, 0.0, 2.0, 4.0, 0.0, 0.0, 0.0]
    s = np.array([1, 2, 2], dtype=np.int64)
    y = SP.real_series(s, 4)
    assert abs(y[:3].sum()) < 1e-15 and y[3] == 0.0


def test_whiten_median_is_ln2_and_noise_mean_one():
    rng = np.random.default_rng(5)
    N = 1 << 16
    y = rng.standard_normal(N) * 3.0 + 0.01 * np.arange(N) / N  # slow trend
    A = SP.half_spectrum(y)
    W = 1024
    Ap = SP.whiten(A, W)
    assert Ap[0] == 0
    p = np.abs(Ap) ** 2
    for b in range(Ap.shape[0] // W):
        blk = p[b * W:(b + 1) * W]
        if b == 0:
            blk = blk[1:]
        assert abs(np.sort(blk)[(blk.shape[0] - 1) // 2] - math.log(2.0)) < 1e-12
    m = p[1:].mean()
    assert abs(m - 1.0) < 3.0 / math.sqrt(p.shape[0])


def test_whiten_zero_block():
    A = np.zeros(2048, dtype=np.complex128)
    A[1500] = 3.0
    Ap = SP.whiten(A, 1024)
    assert np.all(Ap == 0)


def test_whiten_single_block_spectrum():
    # the ds 128 rows of the Table 3 plan: nfft 2048, one block of 1024 bins whose
    # median excludes the zeroed DC bin (1023 values, lower median index 511)
    rng = np.random.default_rng(9)
    y = rng.standard_normal(2048) * 5.0 + 7.0
    A = SP.half_spectrum(y)
    assert A.shape[0] == 1024
    Ap = SP.whiten(A, 1024)
    p = np.abs(Ap) ** 2
    assert p[0] == 0
    assert abs(np.sort(p[1:])[511] - math.log(2.0)) < 1e-12
    # the scale is the one block's: every bin is multiplied by the same factor
    ratio = p[1:] / (np.abs(A[1:]) ** 2)
    assert np.allclose(ratio, ratio[0], rtol=1e-12)
