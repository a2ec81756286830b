"""Pins for the automatic dedispersion plan (oracle/ddplan.py)."""
import math
import os

import pytest

from oracle import ddplan as DP

GOLD = os.path.join(os.path.dirname(__file__), "golden", "ddplan_tables.txt")


def _tables():
    t = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        name, _, lo, hi, step, ds, n = line.split()
        t.setdefault(name, []).append((float(lo), float(hi), float(step), int(ds), int(n)))
    return t


# the two files of the paper's Table 1: PMPS (96 x 3 MHz, 1231.5-1516.5 MHz, 250 us)
# and FAST (200 x 0.25 MHz, 290-340 MHz, 52.4288 s in 2^19 samples: 100 us)
PMPS = dict(fch0=1231.5, foff=3.0, nchan=96, tsamp=250e-6)   # channel centres 1231.5-1516.5
FAST = dict(fch0=290.0 + 0.125, foff=0.25, nchan=200, tsamp=100e-6)


@pytest.mark.parametrize("name,f,kw", [("table2", PMPS, dict(dm_hi=3896.0)),
                                       ("table3", FAST, dict(dm_hi=784.4, tres=0.8e-3, ds_max=128))])
def test_reproduces_the_printed_tables_approximately(name, f, kw):
    ref = _tables()[name]
    rows = DP.auto_plan(f["fch0"], f["foff"], f["nchan"], f["tsamp"], 0.0, **kw)
    # the same downsampling sequence over the printed rows
    assert [r[3] for r in rows[:len(ref)]] == [r[3] for r in ref]
    for (lo, hi, step, ds, n), (d0, s, k, dsx) in zip(ref, rows):
        assert 1 / 2.5 <= s / step <= 2.5, (name, step, s)
        if hi < kw["dm_hi"]:
            assert 1 / 1.7 <= (d0 + k * s) / hi <= 1.7, (name, hi, d0 + k * s)


def test_rows_are_contiguous_cover_the_range_and_obey_the_rule():
    f = PMPS
    rows = DP.auto_plan(f["fch0"], f["foff"], f["nchan"], f["tsamp"], 3.0, 2000.0)
    ctr, dnu, bw = DP.band(f["fch0"], f["foff"], f["nchan"])
    nu = ctr / 1e3
    assert rows[0][0] == 3.0
    for (d0, s, n, ds), nxt in zip(rows, rows[1:] + [None]):
        ts = ds * f["tsamp"]
        T = math.hypot(ts, 8.3e-6 * d0 * dnu / nu ** 3)
        # the half-step smearing fits the resolution; the next listed step does not
        assert 8.3e-6 * (s / 2) * bw / nu ** 3 <= T * (1 + 1e-12)
        i = DP.STEPS.index(s)
        if i + 1 < len(DP.STEPS):
            assert 8.3e-6 * (DP.STEPS[i + 1] / 2) * bw / nu ** 3 > T * (1 - 1e-12)
        if nxt is not None:
            assert nxt[0] == d0 + n * s and nxt[3] == 2 * ds
            # the stage ended where the channel smearing first reaches kappa * ts (to one step)
            end = d0 + n * s
            assert 8.3e-6 * (end - s) * dnu / nu ** 3 < DP.KAPPA * ts * (1 + 1e-12)
    last = rows[-1]
    assert last[0] + last[2] * last[1] >= 2000.0 > last[0]


def test_band_centre_and_width():
    # Table 1: PMPS 1231.5-1516.5 MHz in 96 x 3 MHz channels
    ctr, dnu, bw = DP.band(PMPS["fch0"], PMPS["foff"], 96)
    assert (ctr, dnu, bw) == (1374.0, 3.0, 288.0)
    # a capped downsampling keeps the factor but still changes the step
    rows = DP.auto_plan(FAST["fch0"], FAST["foff"], 200, 100e-6, 0.0, 784.4, tres=0.8e-3, ds_max=128)
    assert [r[3] for r in rows] == [8, 16, 32, 64, 128, 128] and rows[-1][1] > rows[-2][1]
    ctr, dnu, bw = DP.band(340.0 - 0.125, -0.25, 200)   # descending order, same band
    assert (ctr, dnu, bw) == (315.0, 0.25, 50.0)


def test_no_listed_step_fits_takes_the_smallest():
    # a wide low-frequency band sampled at 0.1 us: even the smallest listed
    # step smears by more than the resolution at DM 0, so the first row takes
    # that smallest step
    fch0, foff, nchan, ts = 200.0, 1.0, 200, 1e-7
    ctr, dnu, bw = DP.band(fch0, foff, nchan)
    nu = ctr / 1e3
    assert 8.3e-6 * (DP.STEPS[0] / 2) * bw / nu ** 3 > ts
    rows = DP.auto_plan(fch0, foff, nchan, ts, 0.0, 1.0)
    assert rows[0][1] == DP.STEPS[0] and rows[0][3] == 1
