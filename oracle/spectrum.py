"""Time series -> normalised spectrum (Sect. 2 step 3, realfft).

Mean subtraction, zero padding and whitening are not described in the
paper; the readings below are this project's and are listed with the
design notes.
"""
from __future__ import annotations

import math

import numpy as np


def real_series(s: np.ndarray, nfft: int) -> np.ndarray:
    """FP64 [nfft]: y[n] = s[n] - mean(s) for n < N_v, 0 beyond.

    The mean is the exact integer sum divided by N_v in FP64."""
    nv = int(s.shape[0])
    mu = float(int(np.sum(s, dtype=np.int64))) / float(nv)
    y = np.zeros(nfft, dtype=np.float64)
    y[:nv] = s.astype(np.float64) - mu
    return y


def half_spectrum(y: np.ndarray) -> np.ndarray:
    """complex128 [nfft/2]: A_k = sum_n y_n exp(-2 pi i k n / nfft),
    k = 0 .. nfft/2 - 1 (the Nyquist bin is dropped).  numpy's FFT is a
    library step here; it is pinned against a brute-force DFT."""
    nfft = y.shape[0]
    return np.fft.rfft(y)[: nfft // 2]


def lower_median(v: np.ndarray) -> float:
    """Element of rank floor((m-1)/2) of the sorted values (m = len)."""
    srt = np.sort(np.asarray(v, dtype=np.float64))
    return float(srt[(srt.shape[0] - 1) // 2])


def whiten(A: np.ndarray, block: int = 1024) -> np.ndarray:
    """Block-median normalisation.

    Reading: bins are cut into blocks [b*W, (b+1)*W); the DC bin is set to 0
    and left out of block 0's statistics; med_b is the lower median of
    |A_k|^2 over the block; A'_k = A_k * sqrt(ln 2 / med_b).  For
    exponentially distributed noise power the median is ln 2 times the
    mean, so noise powers come out with mean 1.  A block whose median is 0
    (degenerate input) is set to 0."""
    M = A.shape[0]
    if M % block != 0:
        raise ValueError("spectrum length must be a multiple of the block")
    out = np.array(A, dtype=np.complex128, copy=True)
    out[0] = 0.0
    for b in range(M // block):
        lo = b * block
        seg = out[lo: lo + block]
        p = (seg.real ** 2 + seg.imag ** 2)
        if b == 0:
            p = p[1:]
        med = lower_median(p)
        if med > 0.0:
            out[lo: lo + block] = seg * math.sqrt(math.log(2.0) / med)
        else:
            out[lo: lo + block] = 0.0
    return out
