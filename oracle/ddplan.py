"""Automatic dedispersion plan (DDplan-like stage generation).

TEST INFRASTRUCTURE: like the rest of `oracle/`, only the tests, the smoke
check and the CPU-baseline leg of the benchmark use this module.

The paper generates its plans (Tables 2 and 3) with PRESTO's DDplan.py
(Sect. 3.1) and prints only the resulting rows.  This module's rule is this
project's reading, built from the textbook smearing terms (nu in GHz, band
widths in MHz, times in s):

* channel smearing at DM:            t_chan(DM) = 8.3e-6 * DM * dnu / nu^3
* smearing of a DM error d over the band: t_bw(d) = 8.3e-6 * d * BW / nu^3
  (nu = the band centre, dnu = |foff|, BW = nchan * |foff|).
* The first stage downsamples by the smallest power of two ds with
  ds * tsamp >= tres (at least 1, at most ds_max); each later stage doubles
  a nominal factor v (starting at that ds) and downsamples by min(v, ds_max).
* A stage starting at DM d0 with sampling ts = min(v, ds_max) * tsamp has the
  effective resolution T = sqrt(ts^2 + t_chan(d0)^2); it takes the largest
  step s of the list 1, 2, 3, 5 x 10^k whose half-step smearing t_bw(s/2)
  is at most T (the smallest listed step if none is), and runs
  to the DM where the channel smearing reaches kappa * v * tsamp
  (DM_sw = kappa * v * tsamp / (8.3e-6 * dnu / nu^3)), at least one step and at
  most dm_hi: n = ceil((end - d0) / s - 1e-9) trials, and the next stage
  starts at d0 + n * s.
* kappa = 3.5 (DDplan's own constants are not given in the paper; with
  3.5 the rule reproduces both printed tables' downsampling sequences,
  their steps within a factor 2.5 and their boundaries within a factor 1.7).
"""
from __future__ import annotations

import math

STEPS = (0.01, 0.02, 0.03, 0.05, 0.1, 0.2, 0.3, 0.5, 1.0, 2.0, 3.0, 5.0, 10.0, 20.0, 30.0, 50.0,
         100.0, 200.0, 300.0, 500.0, 1000.0)
KAPPA = 3.5


def band(fch0: float, foff: float, nchan: int):
    """(centre MHz, |foff| MHz, BW MHz)."""
    ctr = fch0 + 0.5 * (nchan - 1) * foff
    return ctr, abs(foff), nchan * abs(foff)


def auto_plan(fch0: float, foff: float, nchan: int, tsamp: float, dm_lo: float, dm_hi: float,
              tres: float = 0.0, ds_max: int = 1024, kappa: float = KAPPA):
    """Rows (dm_lo, dm_step, n_dm, ds) covering [dm_lo, dm_hi)."""
    ctr, dnu, bw = band(fch0, foff, nchan)
    nu = ctr / 1000.0
    kch = 8.3e-6 * dnu / (nu * nu * nu)
    kbw = 8.3e-6 * bw / (nu * nu * nu)
    v = 1
    while v < ds_max and v * tsamp < tres:
        v *= 2
    d0, rows = float(dm_lo), []
    while d0 < dm_hi:
        ds = min(v, ds_max)
        ts = ds * tsamp
        tc = kch * d0
        T = math.sqrt(ts * ts + tc * tc)
        step = STEPS[0]
        for s in STEPS:
            if kbw * (0.5 * s) <= T:
                step = s
        dsw = kappa * (v * tsamp) / kch
        end = min(max(dsw, d0 + step), dm_hi)
        n = max(1, int(math.ceil((end - d0) / step - 1e-9)))
        rows.append((d0, step, n, ds))
        d0 = d0 + n * step
        v *= 2
    return rows
