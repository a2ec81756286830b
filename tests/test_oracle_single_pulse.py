"""Pins for the single-pulse search oracle (oracle/single_pulse.py)."""
import math

import numpy as np
from scipy import stats

from oracle import single_pulse as SP


def _noise(n, seed):
    # a dedispersed series of 256 uint8 channels: integer, close to Gaussian
    rng = np.random.default_rng(seed)
    return np.round(32640 + 256 * rng.standard_normal(n)).astype(np.int64)


def test_moments_match_numpy():
    s = _noise(10007, 1)
    mu, sigma = SP.moments(s)
    assert abs(mu - s.mean()) <= 1e-12 * abs(mu)
    assert abs(sigma - s.std()) <= 1e-9 * sigma


def test_boxcars_brute_force():
    rng = np.random.default_rng(2)
    s = rng.integers(0, 5000, 57)
    for w in (1, 2, 5, 57):
        ref = [sum(int(s[t + k]) for k in range(w)) for t in range(57 - w + 1)]
        assert SP.boxcars(s, w).tolist() == ref


def _brute_detections(s, widths, thr):
    n = len(s)
    mu, sigma = SP.moments(s)
    out = []
    for w in widths:
        if w > n:
            continue
        B = [sum(int(s[t + k]) for k in range(w)) for t in range(n - w + 1)]
        T = float(w) * mu + (thr * sigma) * math.sqrt(float(w))
        for t in range(n - w + 1):
            if not float(B[t]) >= T:
                continue
            ok = all(B[t] > B[u] for u in range(max(0, t - w + 1), t)) and \
                all(B[t] >= B[u] for u in range(t + 1, min(n - w + 1, t + w)))
            if ok:
                out.append((t, w, B[t]))
    return sorted(out)


def test_detections_brute_force():
    s = _noise(400, 3)
    s[100:106] += 900        # a pulse of 6 samples
    s[250] += 2000           # a spike
    s[300:303] = s[299]      # a plateau (ties)
    widths = (1, 2, 3, 6, 9)
    assert sorted(SP.detections(s, widths, 3.0)) == _brute_detections(s, widths, 3.0)


def test_injected_boxcar_is_found_at_its_width_with_matched_filter_snr():
    s = _noise(1 << 15, 4)
    mu0, sig0 = SP.moments(_noise(1 << 15, 4))
    A, w0, t0 = 400, 14, 20000
    s[t0:t0 + w0] += A
    ev = SP.search_series(s, SP.DEFAULT_WIDTHS, 6.0)
    top = max(ev, key=lambda e: e[3])
    t, w, B, sn = top
    assert w == w0 and t == t0
    expect = A * math.sqrt(w0) / sig0            # matched-filter S/N of a boxcar
    assert abs(sn - expect) < 1.5                # noise in the box: about 1 sigma


def test_noise_exceedance_rate_is_the_gaussian_tail():
    # fraction of B_w above the thr-sigma threshold equals Q(thr) for every
    # width (the sqrt(w) normalisation), within 5 binomial sigma
    s = _noise(1 << 18, 5)
    mu, sigma = SP.moments(s)
    q = stats.norm.sf(3.0)
    for w in (1, 4, 20, 100):
        B = SP.boxcars(s, w)
        frac = float(np.mean(B.astype(np.float64) >= SP.threshold(w, mu, sigma, 3.0)))
        n_eff = B.shape[0] / w  # boxcars overlap: about N/w independent values
        assert abs(frac - q) <= 5 * math.sqrt(q * (1 - q) / n_eff), (w, frac, q)


def test_pruning_keeps_the_strongest_non_overlapping():
    mu, sigma = 0.0, 1.0
    dets = [(10, 4, 8), (12, 2, 7), (13, 1, 6), (20, 3, 9), (14, 1, 5)]
    # S/N 4, 4.95, 6, 5.20, 5: kept (13,1), (20,3), (14,1); (12,2) and (10,4) overlap (13,1)
    kept = SP.prune(dets, mu, sigma)
    assert [(t, w) for t, w, _, _ in kept] == [(13, 1), (14, 1), (20, 3)]


def test_constant_series_has_no_events():
    assert SP.search_series(np.full(1000, 77), SP.DEFAULT_WIDTHS, 3.0) == []


def _mean_zero_series(spikes, n_minus, N, seed):
    # n_minus samples of -1 at random places away from the spikes, zeros elsewhere:
    # S1 = 0 exactly when the spikes sum to n_minus, so mu = 0 in FP64
    s = np.zeros(N, dtype=np.int64)
    for t, v in spikes.items():
        s[t] = v
    free = [t for t in range(N) if all(abs(t - u) > 8 for u in spikes)]
    s[np.random.default_rng(seed).choice(free, n_minus, replace=False)] = -1
    assert s.sum() == 0
    return s


def test_a_boxcar_exactly_at_the_threshold_is_detected():
    # 100 samples with S1 = 0 and S2 = 400: mu = 0 and sigma = 2 exactly, so at
    # 5 sigma the one-sample threshold is exactly 10, and a spike of 10 meets it
    vals = [10] + [-3] * 4 + [-1] * 65 + [1] + [3] * 22 + [0] * 7
    s = np.array(vals, dtype=np.int64)
    rest = s[1:].copy()
    np.random.default_rng(3).shuffle(rest)
    s = np.concatenate([rest[:50], [10], rest[50:]])
    mu, sigma = SP.moments(s)
    assert (mu, sigma) == (0.0, 2.0) and SP.threshold(1, mu, sigma, 5.0) == 10.0
    assert SP.detections(s, (1,), 5.0) == [(50, 1, 10)]
    assert SP.detections(s, (1,), math.nextafter(5.0, 6.0)) == []


def test_a_plateau_is_detected_at_its_first_sample():
    # three samples of 10 make two equal neighbouring two-sample boxcars of 20:
    # the left one beats everything to its right (>=) and the right one does
    # not beat it (>), so exactly one event, at the left
    s = _mean_zero_series({100: 10, 101: 10, 102: 10}, 30, 400, 4)
    assert [(t, w) for t, w, _ in SP.detections(s, (2,), 6.0)] == [(100, 2)]


def test_equal_snr_keeps_the_narrower_pulse():
    # 4, 8, 4 around t = 200 with mu = 0: the one-sample boxcar 8 and the
    # four-sample boxcar 16 (t = 198) have the same S/N 8/sigma = 16/(2 sigma)
    # in FP64; they overlap, and the tie goes to the smaller width, after
    # which the one-sample events at 199 and 201 no longer overlap anything kept
    s = _mean_zero_series({199: 4, 200: 8, 201: 4}, 16, 400, 5)
    mu, sigma = SP.moments(s)
    assert mu == 0.0 and SP.snr(8, 1, mu, sigma) == SP.snr(16, 4, mu, sigma)
    assert (198, 4, 16) in SP.detections(s, (1, 4), 6.0)
    ev = SP.search_series(s, (1, 4), 6.0)
    assert [(t, w, B) for t, w, B, _ in ev] == [(199, 1, 4), (200, 1, 8), (201, 1, 4)]
