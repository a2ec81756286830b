"""Pins for the oracle's plan: DM grid and delay table."""
import os

import numpy as np
import pytest

from oracle import plan as P
from paper_1912_12807_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "ddplan_tables.txt")


def _rows():
    rows = {}
    for ln in open(GOLD):
        if ln.startswith("#") or not ln.strip():
            continue
        t, i, lo, hi, step, ds, n = ln.split()
        rows.setdefault(t, []).append((float(lo), float(hi), float(step), int(ds), int(n)))
    return rows


def test_tables_2_3_counts_are_half_open_rows():
    # Paper Tables 2-3: each printed count equals (end - start) / step, so a row
    # is the half-open range [start, end).  The oracle's grid must list exactly
    # that many trials per row, all inside the row.
    rows = _rows()
    assert set(rows) == {"table2", "table3"}
    totals = {}
    for t, rr in rows.items():
        stages = [synth.Stage(lo, step, n, ds) for lo, hi, step, ds, n in rr]
        dms, st, dss = P.dm_grid(stages)
        for k, (lo, hi, step, ds, n) in enumerate(rr):
            assert int(round((hi - lo) / step)) == n
            sel = dms[st == k]
            assert sel.shape[0] == n
            assert sel[0] == lo
            assert np.all(sel < hi - 0.25 * step)
            assert np.all(dss[st == k] == ds)
        totals[t] = dms.shape[0]
    assert totals == {"table2": 789, "table3": 979}


def test_stage_builder_matches_tables():
    rows = _rows()
    for t, rr in rows.items():
        st = synth.stages_from_table([(lo, hi, step, ds) for lo, hi, step, ds, _ in rr], last_inclusive=False)
        assert [s.n_dm for s in st] == [n for *_, n in rr]
    # "DM 0-100 step 1 (101 trials)": the inclusive end of a single-row plan.
    assert synth.stages_from_table([(0.0, 100.0, 1.0, 1)], last_inclusive=True)[0].n_dm == 101


def test_round_half_away():
    x = np.array([0.5, 1.5, 2.5, -0.5, -1.5, 0.49999999999999994, 2.4999999999999996, 3.0, 7.5000000001])
    assert P.round_half_away(x).tolist() == [1, 2, 3, -1, -2, 0, 2, 3, 8]


def test_delay_zero_at_reference_and_linear_in_dm():
    f = P.channel_freqs(64, 1202.34375, 4.6875)
    v = P.delay_values(np.array([0.0, 1.0, 2.0, 37.5]), f, 2e-4)
    assert np.all(v[0] == 0.0)
    assert np.all(v[:, -1] == 0.0)          # highest channel is the reference
    assert np.all(np.diff(v[1]) < 0)         # lower frequency arrives later
    np.testing.assert_allclose(v[2], 2 * v[1], rtol=1e-15)
    np.testing.assert_allclose(v[3], 37.5 * v[1], rtol=1e-14)


def test_delay_cold_plasma_sweep_units():
    # Textbook sweep: 4.148808 ms * DM * (nu_lo/GHz)^-2 - (nu_hi/GHz)^-2).  At DM 500
    # over 1050.78..1449.22 MHz with 0.2 ms sampling this is 4455.24 samples.
    f = np.array([1050.78125, 1449.21875])
    v = P.delay_values(np.array([500.0]), f, 2e-4)[0]
    ms = 4.148808 * 500 * ((f[0] / 1e3) ** -2 - (f[1] / 1e3) ** -2)
    assert abs(v[0] - ms / 0.2) < 1e-6
    assert abs(v[0] - 4455.239) < 1e-3
    assert P.delay_table(np.array([500.0]), f, 2e-4)[0].tolist() == [4455, 0]


@pytest.mark.parametrize("wl", ["small", "drift", "accel", "pmps"])
def test_no_delay_near_half(wl):
    # The rounding of every delay in the standard workloads must not hinge on
    # the last bits of FP64 evaluation order.
    shapes = {
        "small": (64, 2e-4, 1200.0, 1500.0, [synth.Stage(0.0, 1.0, 101, 1)]),
        "drift": (256, 2e-4, 1050.0, 1450.0, [synth.Stage(0.0, 0.5, 1001, 1)]),
        "accel": (256, 2e-4, 1050.0, 1450.0, [synth.Stage(0.0, 1.0, 301, 1)]),
        "pmps": (96, 2.5e-4, 1230.0, 1518.0, synth.stages_from_table(
            [(0.0, 200.0, 0.5, 1), (200.0, 600.0, 1.0, 2), (600.0, 2000.0, 5.0, 4)], True)),
    }
    nchan, ts, lo, hi, stages = shapes[wl]
    fch0, foff = synth.band(lo, hi, nchan)
    dms, _, _ = P.dm_grid(stages)
    v = P.delay_values(dms, P.channel_freqs(nchan, fch0, foff), ts)
    frac = np.abs(v - np.floor(v) - 0.5)
    # DM 0 rows are exactly 0; every other value stays away from .5
    assert frac.min() > 1e-9


def test_channel_centres_tile_the_band():
    # fch0 is the centre of channel 0 (the filterbank header's first-channel
    # frequency), so a descending 3-channel header reads back unchanged ...
    assert P.channel_freqs(3, 1400.0, -1.0).tolist() == [1400.0, 1399.0, 1398.0]
    # ... and n channels of width |foff| laid from the band's lower edge have
    # their edges at lo + c * width: the first starts at lo, the last ends at hi
    for lo, hi, n in ((1200.0, 1500.0, 64), (1050.0, 1450.0, 256), (290.0, 340.0, 200)):
        f = P.channel_freqs(n, *synth.band(lo, hi, n))
        w = (hi - lo) / n
        np.testing.assert_allclose(f - w / 2, lo + np.arange(n) * w, rtol=0, atol=1e-9)
        np.testing.assert_allclose(f + w / 2, lo + np.arange(1, n + 1) * w, rtol=0, atol=1e-9)


def test_stage_lengths():
    assert P.stage_lengths(1 << 18, 4455, 1) == (262144 - 4455, 1 << 18)
    # a valid length that is already a power of two is transformed unpadded
    assert P.stage_lengths((1 << 18) + 4455, 4455, 1) == (1 << 18, 1 << 18)
    assert P.stage_lengths((1 << 18) * 4 + 7, 7, 4) == (1 << 18, 1 << 18)
    assert P.stage_lengths((1 << 18) + 4456, 4455, 1) == ((1 << 18) + 1, 1 << 19)
    assert P.stage_lengths(1 << 23, 7453, 4) == ((8388608 - 7453) // 4, 1 << 21)
    with pytest.raises(ValueError):
        P.stage_lengths(100, 100, 1)


def test_file_shape_sizes():
    # Table 1 / Sect. 1 sizes follow from channels x samples x bits.
    for ln in open(os.path.join(os.path.dirname(__file__), "golden", "file_shapes.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        name, nchan, ts, dur, mb, bits = ln.split()[:6]
        nbytes = int(nchan) * (float(dur) / float(ts)) * int(bits) / 8
        assert abs(nbytes / 1e6 - float(mb)) / float(mb) < 0.15, name


def test_fast_workload_uses_table_3():
    # the FAST-shaped benchmark file is searched with the printed Table 3 plan
    rr = _rows()["table3"]
    assert [tuple(r[:4]) for r in rr] == [tuple(map(float, r[:3])) + (r[3],) for r in synth.TABLE3_ROWS]
    st = synth.stages_from_table(synth.TABLE3_ROWS, last_inclusive=False)
    assert sum(s.n_dm for s in st) == 979 and [s.ds for s in st] == [8, 16, 32, 64, 128, 128]
