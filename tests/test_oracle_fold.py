"""Pins for the folding oracle (oracle/fold.py)."""
import math

import numpy as np
from scipy import stats

from oracle import fold as FO


def test_phase_bins_brute_force():
    # exact rational phases: f = 3/8 Hz, dt = 1/4 s -> phase j*3/32; bins of 8
    b = FO.phase_bins(40, 0.25, 0.375, 0.0, 8)
    ref = [((j * 3) % 32) * 8 // 32 for j in range(40)]
    assert b.tolist() == ref


def test_fold_brute_force_with_drift():
    rng = np.random.default_rng(1)
    s = rng.integers(0, 1000, 500)
    dt, f, fdot, nbin = 1e-3, 37.3, 2.1, 16
    P, n = FO.fold(s, dt, f, fdot, nbin)
    Pr, nr = [0] * nbin, [0] * nbin
    for j in range(500):
        t = j * dt
        ph = f * t + 0.5 * fdot * t * t
        k = int(math.floor((ph - math.floor(ph)) * nbin))
        Pr[k] += int(s[j])
        nr[k] += 1
    assert P.tolist() == Pr and n.tolist() == nr
    assert int(P.sum()) == int(s.sum()) and int(n.sum()) == 500


def test_chi2_of_noise_is_chi2_distributed():
    # white noise folded at an unrelated frequency: chi2 follows chi2(nbin - 1),
    # so chi2_red has mean 1 and sd sqrt(2/(nbin-1)); over 200 folds the mean is 1 +- 5 sd/sqrt(200)
    rng = np.random.default_rng(2)
    nbin, vals = 32, []
    for i in range(200):
        s = np.round(1000 + 30 * rng.standard_normal(4096)).astype(np.int64)
        mu = s.mean()
        var = float(((s - mu) ** 2).mean())
        P, n = FO.fold(s, 1e-3, 7.77 + 0.01 * i, 0.0, nbin)
        vals.append(FO.chi2_red(P, n, float(s.sum()) / 4096, var))
    sd = math.sqrt(2.0 / (nbin - 1))
    assert abs(np.mean(vals) - 1.0) < 5 * sd / math.sqrt(200)
    # and the distribution itself (Kolmogorov-Smirnov against chi2(nbin-1)/(nbin-1))
    p = stats.kstest(np.array(vals) * (nbin - 1), "chi2", args=(nbin - 1,)).pvalue
    assert p > 1e-3


def test_fold_search_finds_the_injected_frequency():
    # a pulse train at f0 = 13.1 Hz folded from a grid started 2 bins off
    rng = np.random.default_rng(3)
    N, dt = 1 << 15, 5e-4
    T = N * dt
    t = np.arange(N) * dt
    f0 = 13.1
    ph = (f0 * t) % 1.0
    s = np.round(1000 + 30 * rng.standard_normal(N) + 40 * (ph < 0.05)).astype(np.int64)
    k, fk, c, P, n = FO.fold_search(s, dt, T, f0 + 2.0 / T, 0.0, 64, 9, 0.5)
    assert k == 0 and abs(fk - f0) < 1e-12            # 2 bins = 4 steps of 0.5 below the centre
    assert c > 20  # about 38 expected: 5 % duty, 1.3 sigma per sample
    assert int(np.argmax(P / n)) in (0, 1, 2, 3)      # the pulse sits at phase 0-0.05
    # the chi2 of a flat series is 0
    assert FO.fold_search(np.full(1000, 5), dt, T, 3.0, 0.0, 16, 3, 1.0)[2] == 0.0


def test_drift_term_realigns_a_chirped_train():
    # a pulse train whose frequency drifts by 3 bins over the span folds sharply
    # only with its fdot (a dropped or wrong-signed drift term smears it)
    rng = np.random.default_rng(4)
    N, dt = 1 << 15, 5e-4
    T = N * dt
    t = np.arange(N) * dt
    f0, fd = 13.1, 3.0 / T / T
    ph = (f0 * t + 0.5 * fd * t * t) % 1.0
    s = np.round(1000 + 30 * rng.standard_normal(N) + 40 * (ph < 0.05)).astype(np.int64)
    good = FO.fold_search(s, dt, T, f0, fd, 64, 1, 0.0)[2]
    none = FO.fold_search(s, dt, T, f0, 0.0, 64, 1, 0.0)[2]
    wrong = FO.fold_search(s, dt, T, f0, -fd, 64, 1, 0.0)[2]
    assert good > 3 * none and good > 3 * wrong


def test_fixed_point_is_the_exact_rounded_fraction():
    # X = rint(v 2^64) mod 2^64 of the exact binary value of v, for either sign and
    # for values whose fraction 1 + v (v < 0) FP64 cannot hold
    from fractions import Fraction
    assert FO.fixed_point(0.25) == 1 << 62 and FO.fixed_point(-0.25) == 3 << 62
    rng = np.random.default_rng(6)
    vals = [-4e-10, 4e-10, -1e-17, -0.5, 0.5, -3.75, 1234.5678, -1234.5678, 2.0 ** -70, -(2.0 ** -70),
            1.0 - 2.0 ** -53, -1.0 + 2.0 ** -53] + list(rng.uniform(-5, 5, 50)) + list(rng.uniform(-1e-9, 1e-9, 50))
    for v in vals:
        want = int(round((Fraction(v) % 1) * 2 ** 64)) % 2 ** 64
        assert FO.fixed_point(float(v)) == want, v


def test_fixed_point_phase_matches_exact_rational_phase():
    # the 64-bit fixed-point bins equal floor(frac(j x + j^2 g) nbin) of the exact
    # rational phase of the FP64 x = f dt and g = (fdot/2) dt^2, except where that
    # phase lies within the fixed-point rounding, (j + j^2) 2^-65 cycle, of a bin
    # edge; drifts of both signs, long series, bin counts that are and are not
    # powers of two
    from fractions import Fraction
    rng = np.random.default_rng(5)
    for it in range(8):
        f, dt = rng.uniform(0.5, 400), rng.uniform(1e-4, 1e-3)
        fd = rng.uniform(-3, 3) if it % 2 else -rng.uniform(1e-3, 0.1)
        nbin = int(rng.integers(2, 100)) if it < 4 else 64
        n = 300000
        got = FO.phase_bins(n, dt, f, fd, nbin)
        x = Fraction(f * dt)
        g = Fraction((0.5 * fd) * (dt * dt))
        for j in list(range(0, 3000, 7)) + list(range(3000, n, 997)):
            ph = (j * x + j * j * g) % 1
            b = int(ph * nbin)
            if b != int(got[j]):
                edge = min(abs(ph * nbin - b), abs(ph * nbin - (b + 1))) / nbin
                assert edge <= Fraction(j + j * j, 2 ** 65), (it, j, b, got[j])


def test_bin_of_phase_is_the_exact_floor_at_every_bin_edge():
    # floor(ph * nbin / 2^64) in exact integers: at the first phase of every bin,
    # one unit below it, and at random phases
    rng = np.random.default_rng(12)
    for nbin in (2, 3, 7, 64, 100, 1000, 1024):
        edges = [-(-(m << 64) // nbin) for m in range(1, nbin)]   # ceil(m 2^64 / nbin)
        ph = edges + [e - 1 for e in edges] + [0, (1 << 64) - 1]
        ph += [int(v) for v in rng.integers(0, 1 << 63, 200, dtype=np.uint64)]
        ph += [int(v) | (1 << 63) for v in rng.integers(0, 1 << 63, 200, dtype=np.uint64)]
        got = FO.bin_of_phase(np.array(ph, dtype=np.uint64), nbin)
        assert got.tolist() == [(p * nbin) >> 64 for p in ph], nbin


def test_reduced_chi2_by_hand():
    # s = 0, 2, 0, 2, ... folded at half the sample rate: even samples fall in
    # bin 0, odd ones in bin nbin/2.  mu = 1, var = 1; each used bin holds 4
    # samples with d = -4 and +4, so chi2 = 16/4 + 16/4 = 8 over 2 used bins:
    # chi2_red = 8 / (2 - 1), whatever the number of empty bins.
    s = np.array([0, 2] * 4)
    for nbin in (2, 4, 16):
        P, n = FO.fold(s, 1.0, 0.5, 0.0, nbin)
        assert n.tolist() == [4 if b in (0, nbin // 2) else 0 for b in range(nbin)]
        assert FO.chi2_red(P, n, 1.0, 1.0) == 8.0


def test_equal_trials_keep_the_first():
    # a constant series has var 0, so every trial scores 0 and the first wins
    dt, T = 1e-3, 1.0
    k, fk, c, _, _ = FO.fold_search(np.full(500, 7), dt, T, 5.0, 0.0, 16, 5, 1.0)
    assert (k, c) == (0, 0.0) and fk == 5.0 - 2.0
