"""Shared helpers for the GPU-vs-oracle parity tests (not collected)."""
from __future__ import annotations

import numpy as np

from oracle import dedisperse as OD
from oracle import harmsum as OH
from oracle import plan as OP
from oracle import response as OR
from oracle import spectrum as OS
from oracle import stats as OST
from oracle import subband as OSB

# Tolerances (normalised powers; candidate exception band).
P_RTOL = 1e-4           # |P_gpu - P_ref| <= P_RTOL * max(P_ref, 1)
SIGMA_BAND = 0.05       # candidates within this many sigma of the threshold may differ
TIE_RTOL = 1e-4         # ... as may ones whose local-max test meets a neighbour this close


def oracle_plane(x_cm, P: OP.Plan, dm_idx: int, cfg, method="direct"):
    ds = int(P.ds_of[dm_idx])
    nv, nfft = P.nv_nfft(dm_idx)
    if P.sub is None:
        s = OD.dedisperse(x_cm, P.delays[dm_idx], P.max_delay, ds)
    else:
        s = OSB.dedisperse_subband(x_cm, P.sub, dm_idx, P.max_delay, ds)
    A = OS.half_spectrum(OS.real_series(s, nfft))
    Ap = OS.whiten(A, cfg.whiten_block)
    plane = OR.power_plane(Ap, cfg.zmax, cfg.dz, cfg.halfwidth_extra, method)
    return s, Ap, plane


def check_powers(gpu: np.ndarray, ref: np.ndarray, what: str):
    gpu = np.asarray(gpu, dtype=np.float64)
    err = np.abs(gpu - ref) / np.maximum(ref, 1.0)
    i = int(np.argmax(err))
    assert err.max() <= P_RTOL, "%s: max rel err %.3g at %d (gpu %.8g ref %.8g)" % (what, err.max(), i, gpu.flat[i], ref.flat[i])
    return float(err.max())


def compare_candidates(gpu_rows, plane, dm_idx: int, numharm: int, Z: int, t_span: float, f_lo: float,
                       sigma_thr: float):
    """Compare the GPU raw candidates of one DM trial with the oracle's.

    Exact set equality of (n, h, j) except for points whose oracle S_n is
    within SIGMA_BAND of the threshold or whose local-maximum test meets a
    neighbour within TIE_RTOL; returns (n_gpu, n_ref, n_excused)."""
    thr = OST.thresholds(numharm, sigma_thr)
    ref = {}
    sums = {}
    for n in OST.harmonic_stages(numharm):
        S = OH.harmonic_sum(plane, n, Z)
        sums[n] = S
    for n, h, j, S in OH.raw_candidates(plane, numharm, Z, thr, t_span, f_lo):
        ref[(n, h, j)] = S
    got = {}
    for r in gpu_rows:
        if int(r["dm_idx"]) != dm_idx:
            continue
        got[(int(r["numharm"]), int(r["h"]), int(r["j"]))] = float(r["power"])

    def excused(key):
        n, h, j = key
        S = sums[n]
        s = S[j, h]
        if abs(OST.sigma_of(n, s) - sigma_thr) < SIGMA_BAND:
            return True
        nz, H = S.shape
        for dj in (-1, 0, 1):
            for dh in (-1, 0, 1):
                if (dj, dh) == (0, 0):
                    continue
                jj, hh = j + dj, h + dh
                if 0 <= jj < nz and 0 <= hh < H and abs(S[jj, hh] - s) <= TIE_RTOL * s:
                    return True
        return False

    bad = []
    exc = 0
    for k in set(ref) ^ set(got):
        if excused(k):
            exc += 1
        else:
            bad.append((k, ref.get(k), got.get(k)))
    assert not bad, "DM %d: %d unexplained differences, e.g. %s" % (dm_idx, len(bad), bad[:5])
    for k in set(ref) & set(got):
        # S_n sums n powers, each within P_RTOL * max(P, 1)
        assert abs(got[k] - ref[k]) <= P_RTOL * (ref[k] + k[0]), (dm_idx, k, got[k], ref[k])
    return len(got), len(ref), exc
