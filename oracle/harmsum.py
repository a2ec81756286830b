"""Harmonic summing, thresholding and local-maximum selection.

The paper's periodicity search (Sect. 2 step 4, accelsearch) sums
harmonics without stating how.  Reading used here:

* The plane point (h, j) is taken as the n-th harmonic of a fundamental at
  r = h / (2n) bins and z = (j - Z) dz / n (Z = zmax/dz is the z = 0 row).
* Its k-th harmonic (k = 1..n) sits at half-bin
      h_k = floor((2 k h + n) / (2 n))      (k h / n rounded half up)
  and row
      j_k = Z + sgn(j - Z) floor((2 k |j - Z| + n) / (2 n)),
  so every index is an exact integer and rounding is symmetric in +-z.
* S_n(h, j) = sum_{k=1..n} P[j_k][h_k] for n in {1, 2, 4, ..., numharm}.
* A raw candidate of stage n is a point with S_n >= S_thr(n), fundamental
  frequency h / (2 n T) >= f_lo, and S_n strictly above each of its (up
  to 8) in-plane neighbours at the same stage; an exact tie is won by the
  lower linear index j * nfft + h.
"""
from __future__ import annotations

import math

import numpy as np

from .stats import harmonic_stages


def harmonic_half_bin(h, k: int, n: int):
    return (2 * k * np.asarray(h, dtype=np.int64) + n) // (2 * n)


def harmonic_row(j, k: int, n: int, Z: int):
    d = np.asarray(j, dtype=np.int64) - Z
    return Z + np.sign(d) * ((2 * k * np.abs(d) + n) // (2 * n))


def harmonic_sum(P: np.ndarray, n: int, Z: int) -> np.ndarray:
    """FP64 [n_z][nfft] of S_n over the whole plane P [n_z][nfft]."""
    nz, H = P.shape
    h = np.arange(H, dtype=np.int64)
    j = np.arange(nz, dtype=np.int64)
    S = np.zeros((nz, H), dtype=np.float64)
    for k in range(1, n + 1):
        hk = harmonic_half_bin(h, k, n)
        jk = harmonic_row(j, k, n, Z)
        S += P[jk][:, hk]
    return S


def local_max(S: np.ndarray) -> np.ndarray:
    """Boolean mask: strictly greater than every in-plane neighbour in the
    3x3 window, exact ties resolved toward the lower linear index."""
    nz, H = S.shape
    idx = np.arange(nz * H, dtype=np.int64).reshape(nz, H)
    keep = np.ones((nz, H), dtype=bool)
    for dj in (-1, 0, 1):
        for dh in (-1, 0, 1):
            if dj == 0 and dh == 0:
                continue
            j0, j1 = max(0, -dj), min(nz, nz - dj)
            h0, h1 = max(0, -dh), min(H, H - dh)
            if j1 <= j0 or h1 <= h0:
                continue
            me = S[j0:j1, h0:h1]
            nb = S[j0 + dj:j1 + dj, h0 + dh:h1 + dh]
            my_i = idx[j0:j1, h0:h1]
            nb_i = idx[j0 + dj:j1 + dj, h0 + dh:h1 + dh]
            wins = (me > nb) | ((me == nb) & (my_i < nb_i))
            keep[j0:j1, h0:h1] &= wins
    return keep


def min_half_bin(n: int, t_span: float, f_lo_hz: float) -> int:
    """Smallest h whose fundamental h/(2 n T) is >= f_lo, computed as
    ceil((2n) * T * f_lo) in FP64, left to right."""
    return int(math.ceil(float(2 * n) * t_span * f_lo_hz))


def raw_candidates(P: np.ndarray, numharm: int, Z: int, thr: dict,
                   t_span: float, f_lo_hz: float, sums: dict = None):
    """List of (n, h, j, S_n) for every stage, in (n, j, h) order.  `sums`
    may hold S_n of some stages already computed by harmonic_sum(P, n, Z)."""
    out = []
    for n in harmonic_stages(numharm):
        S = sums[n] if sums is not None and n in sums else harmonic_sum(P, n, Z)
        m = (S >= thr[n]) & local_max(S)
        hmin = min_half_bin(n, t_span, f_lo_hz)
        if hmin > 0:
            m[:, :hmin] = False
        jj, hh = np.nonzero(m)
        for j, h in zip(jj.tolist(), hh.tolist()):
            out.append((n, h, j, float(S[j, h])))
    return out
