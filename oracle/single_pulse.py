"""Single-pulse (boxcar matched-filter) search of a dedispersed series.

TEST INFRASTRUCTURE: like the rest of `oracle/`, only the tests, the smoke
check and the CPU-baseline leg of the benchmark use this module.

The paper's pipeline ends with a single-pulse search of the dedispersed
series (single_pulse_search.py, Sect. 2 step 7), and notes that the
long-period pulsars its 52 s drift scans miss were found by a single-pulse
search (Sect. 5.3).  It gives no algorithm; the reading used here:

* Normalisation: with N = N_v samples, S1 = sum s and S2 = sum s^2 (exact
  integers), mu = S1 / N and sigma = sqrt((S2 - S1*S1/N) / N), FP64 in that
  order, over the whole series.
* Boxcars: for each width w of the list, B_w[t] = sum_{k<w} s[t+k] for
  0 <= t <= N - w (exact integers); S/N = (B_w[t] - w*mu) / (sigma*sqrt(w)).
* Detection: B_w[t] >= w*mu + thr*sigma*sqrt(w) (the FP64 threshold,
  evaluated in that order), and B_w[t] is a local maximum over a window of
  its own width: B_w[t] > B_w[t'] for t - w < t' < t and B_w[t] >= B_w[t']
  for t < t' < t + w (t' in range).  Both tests are exact: integers against
  one FP64 number per (trial, width).
* Pruning, per trial: the detections ordered by S/N (descending; ties:
  smaller w, then smaller t) are kept one by one when their interval
  [t, t + w) overlaps no interval kept before.  A constant series (sigma 0)
  has no detections.
"""
from __future__ import annotations

import math
from typing import List, Tuple

import numpy as np

DEFAULT_WIDTHS = (1, 2, 3, 4, 6, 9, 14, 20, 30, 45, 70, 100, 150)


def moments(s: np.ndarray) -> Tuple[float, float]:
    """(mu, sigma) of the whole series (module docstring)."""
    s = np.asarray(s, dtype=np.int64)
    n = s.shape[0]
    S1 = int(s.sum())
    S2 = int((s * s).sum())
    fS1, fS2, fN = float(S1), float(S2), float(n)
    mu = fS1 / fN
    var = (fS2 - fS1 * fS1 / fN) / fN
    return mu, math.sqrt(max(var, 0.0))


def threshold(w: int, mu: float, sigma: float, thr: float) -> float:
    """w*mu + thr*sigma*sqrt(w) in FP64, in that order."""
    return float(w) * mu + (thr * sigma) * math.sqrt(float(w))


def boxcars(s: np.ndarray, w: int) -> np.ndarray:
    """int64 [N - w + 1]: B_w[t] = sum_{k<w} s[t+k], from a prefix sum."""
    c = np.concatenate([[0], np.cumsum(np.asarray(s, dtype=np.int64))])
    return c[w:] - c[:-w]


def detections(s: np.ndarray, widths, thr: float) -> List[Tuple[int, int, int]]:
    """(t, w, B) of every detection before pruning (module docstring)."""
    mu, sigma = moments(s)
    if sigma <= 0.0:
        return []
    out = []
    for w in widths:
        w = int(w)
        if w > s.shape[0]:
            continue
        B = boxcars(s, w)
        T = threshold(w, mu, sigma, thr)
        for t in np.nonzero(B.astype(np.float64) >= T)[0]:
            t = int(t)
            lo, hi = max(0, t - w + 1), min(B.shape[0], t + w)
            left = B[lo:t]
            right = B[t + 1:hi]
            if (left.size == 0 or B[t] > left.max()) and (right.size == 0 or B[t] >= right.max()):
                out.append((t, w, int(B[t])))
    return out


def snr(B: int, w: int, mu: float, sigma: float) -> float:
    """(B - w*mu) / (sigma*sqrt(w)) in FP64, in that order."""
    return (float(B) - float(w) * mu) / (sigma * math.sqrt(float(w)))


def prune(dets, mu: float, sigma: float):
    """Greedy non-overlap pruning (module docstring); returns (t, w, B, snr)
    sorted by t."""
    scored = sorted(((snr(B, w, mu, sigma), t, w, B) for t, w, B in dets), key=lambda e: (-e[0], e[2], e[1]))
    kept = []
    for sn, t, w, B in scored:
        if all(t + w <= kt or kt + kw <= t for kt, kw, _, _ in kept):
            kept.append((t, w, B, sn))
    return sorted(kept)


def search_series(s: np.ndarray, widths=DEFAULT_WIDTHS, thr: float = 6.0):
    """Pruned single-pulse events of one dedispersed series: (t, w, B, snr)."""
    mu, sigma = moments(s)
    return prune(detections(s, widths, thr), mu, sigma)
