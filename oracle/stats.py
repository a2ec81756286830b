"""Detection statistics for harmonic-summed powers.

The paper thresholds candidates through accelsearch's sigma without
stating it.  Reading: normalised noise powers are Exp(1), so a sum of n
independent ones is Gamma(n, 1); its tail probability is
    p = Q(n, S) = exp(-S) * sum_{j<n} S^j / j!     (integer n),
and sigma is the single-trial Gaussian equivalent Phi^-1(1 - p).  No
trials-factor correction is applied.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def log_q(n: int, S: float) -> float:
    """log Q(n, S) by a log-sum-exp over the n Poisson terms."""
    if S <= 0.0:
        return 0.0
    lS = math.log(S)
    terms = [j * lS - S - math.lgamma(j + 1) for j in range(int(n))]
    mx = max(terms)
    return mx + math.log(sum(math.exp(t - mx) for t in terms))


def sigma_of(n: int, S: float) -> float:
    """Gaussian-equivalent significance of a harmonic sum S over n terms."""
    return float(-special.ndtri_exp(log_q(n, S)))


def power_threshold(n: int, sigma: float) -> float:
    """The S at which sigma_of(n, S) equals sigma, by bisection (60 halvings
    of a bracket that always contains it)."""
    lo, hi = 0.0, 10.0
    while sigma_of(n, hi) < sigma:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if sigma_of(n, mid) < sigma:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-13 * hi:
            break
    return hi


def thresholds(numharm: int, sigma: float):
    return {n: power_threshold(n, sigma) for n in harmonic_stages(numharm)}


def harmonic_stages(numharm: int):
    if numharm < 1 or (numharm & (numharm - 1)) != 0:
        raise ValueError("numharm must be a power of two")
    out, n = [], 1
    while n <= numharm:
        out.append(n)
        n *= 2
    return out
