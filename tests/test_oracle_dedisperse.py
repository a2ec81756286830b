"""Pins for the oracle's dedispersion and channel unpacking."""
import numpy as np

from oracle import dedisperse as DD
from oracle import plan as P
from paper_1912_12807_gb300 import synth


def _brute(x, d, D, ds, mask=None):
    # Pure-Python triple loop over (t, c) then boxcar.
    C, N = x.shape
    L = N - D
    s = [0] * L
    for t in range(L):
        acc = 0
        for c in range(C):
            if mask is None or mask[c]:
                acc += int(x[c][t + int(d[c])])
        s[t] = acc
    nv = L // ds
    return [sum(s[j * ds + k] for k in range(ds)) for j in range(nv)]


def test_brute_force_tiny():
    rng = np.random.default_rng(3)
    for ds in (1, 2, 3):
        x = rng.integers(0, 256, size=(7, 53)).astype(np.uint8)
        d = rng.integers(0, 9, size=7)
        D = 11
        mask = [True, False, True, True, True, False, True]
        assert DD.dedisperse(x, d, D, ds).tolist() == _brute(x, d, D, ds)
        assert DD.dedisperse(x, d, D, ds, mask).tolist() == _brute(x, d, D, ds, mask)


def test_total_equals_window_sums():
    # sum_t s[t] = sum_c (sum of x[c] over the window [d_c, d_c + N - D)),
    # computed independently from prefix sums.
    rng = np.random.default_rng(4)
    x = rng.integers(0, 256, size=(32, 4096)).astype(np.uint8)
    d = rng.integers(0, 300, size=32)
    D = 400
    s = DD.dedisperse(x, d, D, 1)
    cs = np.concatenate([np.zeros((32, 1), np.int64), np.cumsum(x.astype(np.int64), axis=1)], axis=1)
    L = 4096 - D
    ref = sum(int(cs[c, d[c] + L] - cs[c, d[c]]) for c in range(32))
    assert int(s.sum()) == ref


def test_wide_downsampling_equals_channel_window_sums():
    # s_ds[j] = sum_c (x[c][j ds + d_c] + ... + x[c][j ds + d_c + ds - 1]): each
    # output is one window sum per channel, taken here from per-channel prefix
    # sums (an order of operations independent of the shift-and-sum)
    rng = np.random.default_rng(8)
    C, N, D = 16, 6000, 700
    x = rng.integers(0, 256, size=(C, N)).astype(np.uint8)
    d = rng.integers(0, D + 1, size=C)
    d[0] = D
    cs = np.concatenate([np.zeros((C, 1), np.int64), np.cumsum(x.astype(np.int64), axis=1)], axis=1)
    for ds in (8, 64, 256):
        nv = (N - D) // ds
        j = np.arange(nv)
        ref = np.zeros(nv, np.int64)
        for c in range(C):
            t = j * ds + d[c]
            ref += cs[c, t + ds] - cs[c, t]
        assert np.array_equal(DD.dedisperse(x, d, D, ds), ref)


def test_one_bit_unpack_msb_first():
    data = np.array([[0b10000000, 0b00000001], [0b01000000, 0b10000000]], dtype=np.uint8)
    x = DD.channel_major(data, 16, 1)
    assert x[:, 0].tolist() == [1] + [0] * 14 + [1]
    assert x[:, 1].tolist() == [0, 1] + [0] * 6 + [1] + [0] * 7
    fil = synth.make_1bit(16, 64, 2.5e-4, 1230.0, 1518.0, [], seed=1)
    assert np.array_equal(DD.channel_major(fil.data, 16, 1), synth.unpack_bits(fil).T)


def test_injected_pulse_realigns_at_its_dm():
    # A narrow dispersed pulse (simulated with continuous delays) lines up in
    # one output sample only at the trial nearest its DM.
    nchan, N, ts = 64, 1 << 14, 2e-4
    fil = synth.make_8bit(nchan, N, ts, 1200.0, 1500.0,
                          [synth.Pulsar(1.0, 60.0, 0.0004, 40.0, phase0=0.5)], seed=9)
    stages = [synth.Stage(40.0, 1.0, 41, 1)]
    pl = P.Plan.for_file(fil, stages)
    x = DD.channel_major(fil.data, nchan, 8)
    peaks = [DD.dedisperse(x, pl.delays[i], pl.max_delay, 1).max() for i in range(len(pl.dms))]
    assert abs(pl.dms[int(np.argmax(peaks))] - 60.0) <= 1.0
