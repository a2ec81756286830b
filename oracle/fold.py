"""Folding of a candidate's dedispersed series (the prepfold step).

TEST INFRASTRUCTURE: like the rest of `oracle/`, only the tests, the smoke
check and the CPU-baseline leg of the benchmark use this module.

The paper folds every sifted candidate at its period and DM with prepfold
(Sect. 2 step 6).  It gives no formulas; the reading used here folds the
candidate's own dedispersed series (its DM trial) and searches a small grid
of trial frequencies around the candidate's:

* Sample j of a series with ds-fold downsampling is at t_j = j * dt,
  dt = ds * tsamp.  Its phase at frequency f and drift fdot (Hz/s) is
  phi_j = f*t_j + (fdot/2)*t_j^2 = j*x + j^2*g cycles, x = f*dt and
  g = (0.5*fdot)*(dt*dt) (FP64, in that order).  The phase is carried in
  64-bit fixed point (units of 2^-64 cycle, wrapping modulo one cycle):
  X = rint(x * 2^64) mod 2^64 and Gq = rint(g * 2^64) mod 2^64 (round half
  to even, on the exact binary values of x and g; a negative value wraps),
  phase_j = (j*X + j*j*Gq) mod 2^64, and the bin is
  floor(phase_j * nbin / 2^64), the fraction of the cycle times nbin
  rounded down, in integers.  The rounding of X and Gq is the only
  departure from the exact phase j*x + j^2*g: at most (j + j^2) 2^-65
  cycle.
* Profile P_b = sum of s_j over the samples of bin b, n_b their number
  (exact integers).
* Significance: with mu = S1/N and var = (S2 - S1*S1/N)/N of the series
  (as in the single-pulse search), chi2 = sum over bins b = 0, 1, ... with
  n_b > 0 of d*d / (n_b*var), d = P_b - n_b*mu, accumulated in bin order;
  chi2_red = chi2 / (number of such bins - 1).  var 0 gives chi2_red 0.
* Trial frequencies f_k = f + (k - (nfreq - 1)/2) * (step / T), T = the
  series span nfft*ds*tsamp of the candidate's trial, k < nfreq; the
  folded result is the trial with the largest chi2_red (ties: smaller k).
"""
from __future__ import annotations

import math

import numpy as np


MASK64 = (1 << 64) - 1


def fixed_point(v: float) -> int:
    """rint(v * 2^64) modulo 2^64, round half to even, exactly: v - trunc(v)
    is exact in FP64 (the integer part is removed without rounding), and so
    is its scaling by 2^64."""
    fr = v - math.trunc(v)
    return int(round(math.ldexp(fr, 64))) & MASK64


def bin_of_phase(ph: np.ndarray, nbin: int) -> np.ndarray:
    """int64: floor(ph * nbin / 2^64) of uint64 phases, exactly, from the two
    32-bit halves of ph (nbin <= 2^10, so no product exceeds 2^42)."""
    hi, lo = ph >> np.uint64(32), ph & np.uint64(0xFFFFFFFF)
    nb = np.uint64(nbin)
    return ((hi * nb + ((lo * nb) >> np.uint64(32))) >> np.uint64(32)).astype(np.int64)


def phase_bins(n: int, dt: float, f: float, fdot: float, nbin: int) -> np.ndarray:
    """int64 [n]: the bin of every sample (module docstring)."""
    X = np.uint64(fixed_point(f * dt))
    G = np.uint64(fixed_point((0.5 * fdot) * (dt * dt)))
    j = np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ph = j * X + (j * j) * G          # uint64 arithmetic wraps modulo 2^64
    return bin_of_phase(ph, nbin)


def fold(s: np.ndarray, dt: float, f: float, fdot: float, nbin: int):
    """(P int64 [nbin], n int64 [nbin]) of one series."""
    b = phase_bins(s.shape[0], dt, f, fdot, nbin)
    P = np.zeros(nbin, dtype=np.int64)
    np.add.at(P, b, np.asarray(s, dtype=np.int64))
    cnt = np.bincount(b, minlength=nbin).astype(np.int64)
    return P, cnt


def chi2_red(P, cnt, mu: float, var: float) -> float:
    """Reduced chi-square of a profile against a flat one (module docstring)."""
    if not var > 0.0:
        return 0.0
    acc, used = 0.0, 0
    for b in range(len(P)):
        nb = int(cnt[b])
        if nb == 0:
            continue
        d = float(int(P[b])) - float(nb) * mu
        acc += d * d / (float(nb) * var)
        used += 1
    return acc / float(used - 1) if used > 1 else 0.0


def trial_freqs(f: float, nfreq: int, step_bins: float, T: float):
    return [f + (float(k) - float(nfreq - 1) / 2.0) * (step_bins / T) for k in range(nfreq)]


def fold_search(s: np.ndarray, dt: float, T: float, f: float, fdot: float, nbin: int, nfreq: int,
                step_bins: float):
    """(best k, f_k, chi2_red, P, n) over the trial frequencies."""
    s64 = np.asarray(s, dtype=np.int64)
    fS1, fS2, fN = float(int(s64.sum())), float(int((s64 * s64).sum())), float(s64.shape[0])
    mu = fS1 / fN
    var = (fS2 - fS1 * fS1 / fN) / fN
    if not var > 0.0:
        var = 0.0
    best = None
    for k, fk in enumerate(trial_freqs(f, nfreq, step_bins, T)):
        P, cnt = fold(s, dt, fk, fdot, nbin)
        c = chi2_red(P, cnt, mu, var)
        if best is None or c > best[2]:
            best = (k, fk, c, P, cnt)
    return best
