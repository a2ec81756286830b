"""Pins for harmonic summing, local maxima, statistics and sifting."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import special, stats as sst

from oracle import harmsum as HS
from oracle import response as R
from oracle import sift as SF
from oracle import spectrum as SP
from oracle import stats as ST


def _round_half_up(fr: Fraction) -> int:
    return math.floor(fr + Fraction(1, 2))


def test_harmonic_indices_exact_rationals():
    for n in (1, 2, 4, 8, 16):
        for h in range(0, 300, 7):
            for k in range(1, n + 1):
                assert int(HS.harmonic_half_bin(h, k, n)) == _round_half_up(Fraction(k * h, n))
        Z = 50
        for j in range(0, 101, 3):
            for k in range(1, n + 1):
                d = j - Z
                ref = Z + (1 if d > 0 else -1 if d < 0 else 0) * _round_half_up(Fraction(k * abs(d), n))
                assert int(HS.harmonic_row(j, k, n, Z)) == ref


def test_harmonic_sum_brute_tiny():
    rng = np.random.default_rng(1)
    P = rng.exponential(size=(9, 40))
    Z = 4
    for n in (1, 2, 4, 8):
        S = HS.harmonic_sum(P, n, Z)
        for j in range(9):
            for h in range(40):
                acc = 0.0
                for k in range(1, n + 1):
                    hk = _round_half_up(Fraction(k * h, n))
                    d = j - Z
                    jk = Z + (d > 0) * _round_half_up(Fraction(k * d, n)) - (d < 0) * _round_half_up(Fraction(-k * d, n))
                    acc += P[jk, hk]
                assert abs(S[j, h] - acc) < 1e-12
    np.testing.assert_array_equal(HS.harmonic_sum(P, 1, Z), P)


def test_local_max_brute_tiny():
    rng = np.random.default_rng(2)
    S = rng.integers(0, 4, size=(5, 12)).astype(float)  # many exact ties
    m = HS.local_max(S)
    nz, H = S.shape
    for j in range(nz):
        for h in range(H):
            ok = True
            for dj in (-1, 0, 1):
                for dh in (-1, 0, 1):
                    if (dj, dh) == (0, 0):
                        continue
                    jj, hh = j + dj, h + dh
                    if 0 <= jj < nz and 0 <= hh < H:
                        me, nb = S[j, h], S[jj, hh]
                        if not (me > nb or (me == nb and j * H + h < jj * H + hh)):
                            ok = False
            assert m[j, h] == ok


def test_pulse_train_harmonic_powers():
    # A Gaussian pulse train of rms phase width s has harmonic amplitudes
    # proportional to exp(-2 pi^2 k^2 s^2): the powers fall as exp(-4 pi^2 k^2 s^2).
    N, nper, duty = 1 << 15, 256, 0.05
    s = duty / 2.3548200450309493
    t = np.arange(N)
    ph = (t * nper / N) % 1.0
    d = ph - np.floor(ph + 0.5)
    y = np.exp(-0.5 * (d / s) ** 2)
    y = y - y.mean()
    A = SP.half_spectrum(y)
    pk = np.array([abs(A[k * nper]) ** 2 for k in range(1, 9)])
    ref = np.exp(-4 * math.pi ** 2 * (np.arange(1, 9) ** 2) * s * s)
    np.testing.assert_allclose(pk / pk[0], ref / ref[0], rtol=1e-6)
    # S_n of the noise-free signal at the n-th harmonic's half-bin equals the sum
    P = (np.abs(A) ** 2)
    row = np.repeat(P, 2)[None, :]  # stand-in plane with P at half-bins 2k, 2k+1
    for n in (1, 2, 4, 8):
        S = HS.harmonic_sum(row, n, 0)
        assert abs(S[0, 2 * n * nper] - pk[:n].sum()) < 1e-9 * pk.sum()


def test_q_function_and_sigma():
    for n in (1, 2, 4, 8, 16):
        for S in (0.5, 3.0, 20.0, 52.0, 150.0):
            lq = ST.log_q(n, S)
            assert abs(lq - math.log(sst.poisson.cdf(n - 1, S))) < 1e-9 * max(1.0, abs(lq)) or S > 100
            assert abs(math.exp(lq) - special.gammaincc(n, S)) <= 1e-12 * max(special.gammaincc(n, S), 1e-300) + 1e-300
    # n = 1: p = exp(-S) exactly
    for S in (0.1, 5.0, 40.0):
        assert abs(ST.log_q(1, S) + S) < 1e-12
    # sigma of the Gaussian tail probability of 6 sigma is 6
    S6 = -math.log(special.ndtr(-6.0))
    assert abs(ST.sigma_of(1, S6) - 6.0) < 1e-9
    assert abs(ST.power_threshold(1, 6.0) - S6) < 1e-9


def test_threshold_table():
    thr = ST.thresholds(16, 6.0)
    for n, v in {1: 20.7368, 2: 23.9538, 4: 29.1688, 8: 37.8435, 16: 52.6057}.items():
        assert abs(thr[n] - v) < 2e-4
        assert abs(ST.sigma_of(n, thr[n]) - 6.0) < 1e-9
    # the stages double: a 16-harmonic search sums 1, 2, 4, 8 and 16 harmonics, no others
    assert sorted(thr) == [1, 2, 4, 8, 16]
    for bad in (0, 3, 12):
        with pytest.raises(ValueError):
            ST.harmonic_stages(bad)


def test_threshold_is_inclusive():
    # a peak whose S_1 equals the threshold exactly is a candidate; one ulp below is not
    thr = {1: 25.0}
    for v, want in ((25.0, [(1, 300, 0)]), (np.nextafter(25.0, 0.0), [])):
        P = np.full((1, 1024), 1.0)
        P[0, 300] = v
        c = HS.raw_candidates(P, 1, 0, thr, 10.0, 0.0)
        assert [(n, h, j) for n, h, j, _ in c] == want


def test_min_half_bin():
    T = 52.4288
    assert HS.min_half_bin(1, T, 1.0) == 105
    assert HS.min_half_bin(4, T, 1.0) == 420
    assert HS.min_half_bin(1, T, 0.0) == 0


def _c(dm, n, r, z, sigma):
    return dict(dm_idx=dm, numharm=n, r=r, z=z, sigma=sigma, h=0, j=0, power=0.0)


def test_sift_hand_built():
    # Within one DM: a chain 100.0 - 100.9 - 101.8 links into one group
    # (single linkage); 110 stays alone; z too far apart does not link.
    c = [_c(0, 1, 100.0, 0.0, 7.0), _c(0, 2, 100.9, 0.0, 9.0), _c(0, 4, 101.8, 0.0, 8.0),
         _c(0, 1, 110.0, 0.0, 6.5), _c(0, 1, 110.0, 10.0, 6.6)]
    w = SF.sift_within(c, 2.0)
    got = sorted((x["r"], x["z"], x["numharm"]) for x in w)
    assert got == [(100.9, 0.0, 2), (110.0, 0.0, 1), (110.0, 10.0, 1)]
    # ties in sigma -> lower n, then lower r
    w = SF.sift_within([_c(0, 4, 50.0, 0.0, 8.0), _c(0, 2, 50.5, 0.0, 8.0)], 2.0)
    assert w[0]["numharm"] == 2
    # Across DMs: the same signal at 3 DMs merges, dm_hits = 3; a lone one stays
    raw = {0: [_c(0, 1, 200.0, 0.0, 7.0)], 1: [_c(1, 1, 200.2, 0.0, 9.0)],
           2: [_c(2, 1, 199.9, 2.0, 8.0)], 3: [_c(3, 1, 500.0, 0.0, 6.1)]}
    out = SF.sift(raw, 2.0, 1)
    assert [(o["dm_idx"], o["dm_hits"]) for o in out] == [(1, 3), (3, 1)]
    out = SF.sift(raw, 2.0, 2)
    assert [(o["dm_idx"], o["dm_hits"]) for o in out] == [(1, 3)]


def test_raw_candidates_noise_false_alarm_rate():
    # Pure Exp(1) powers: the number of 6-sigma single-harmonic peaks is
    # consistent with p(6 sigma) * points (expected 0 here), while a planted
    # peak is found at its position.
    rng = np.random.default_rng(11)
    P = rng.exponential(size=(1, 1 << 16))
    P[0, 5001] = 40.0
    thr = ST.thresholds(1, 6.0)
    c = HS.raw_candidates(P, 1, 0, thr, 10.0, 0.0)
    assert [(n, h, j) for n, h, j, _ in c] == [(1, 5001, 0)]
