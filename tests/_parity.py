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
    for n, h, j, S in OH.raw_candidates(plane, numharm, Z, thr, t_span, f_lo, sums=sums):
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


def oracle_plane_points(Ap: np.ndarray, zmax: int, dz: float, extra: int, js, hs) -> np.ndarray:
    """FP64 powers of the plane at the points (j, h), one by one from the
    definition (the direct sum over the 2m taps nearest r = h/2 at
    z_j = -zmax + j dz, unit-energy normalised, bins outside the spectrum
    zero): for planes too large for the oracle to compute whole."""
    js = np.asarray(js, dtype=np.int64)
    hs = np.asarray(hs, dtype=np.int64)
    zs = OR.z_values(zmax, dz)
    M = Ap.shape[0]
    out = np.empty(js.shape[0], dtype=np.float64)
    for j in np.unique(js):
        for parity in (0, 1):
            sel = np.nonzero((js == j) & (hs % 2 == parity))[0]
            if sel.size == 0:
                continue
            t, g, E = OR.taps(float(zs[j]), parity, extra)
            k = (hs[sel] // 2)[:, None] + t[None, :]
            ok = (k >= 0) & (k < M)
            a = np.where(ok, Ap[np.clip(k, 0, M - 1)], 0.0)
            acc = a @ g
            out[sel] = (acc.real ** 2 + acc.imag ** 2) / E
    return out


def check_candidates_at_points(gpu_rows, Ap, dm_idx: int, numharm: int, zmax: int, dz: float, extra: int,
                               nz: int, nfft: int, t_span: float, f_lo: float, sigma_thr: float):
    """Every GPU raw candidate of one trial, checked against the oracle's
    plane evaluated at just the points its decision needs: S_n at the point
    and at its 8 neighbours (n plane values each).  The candidate's S_n must
    match within the power tolerance, lie above the threshold (or within
    SIGMA_BAND of it) and be a 3x3 local maximum (or tie within TIE_RTOL),
    and its fundamental must be >= f_lo.  Returns the number checked."""
    Z = int(round(zmax / dz)) if zmax else 0
    thr = OST.thresholds(numharm, sigma_thr)
    rows = [r for r in gpu_rows if int(r["dm_idx"]) == dm_idx]
    if not rows:
        return 0
    pts_j, pts_h, owners = [], [], []
    for ci, r in enumerate(rows):
        n, h, j = int(r["numharm"]), int(r["h"]), int(r["j"])
        for dj in (-1, 0, 1):
            for dh in (-1, 0, 1):
                jj, hh = j + dj, h + dh
                if not (0 <= jj < nz and 0 <= hh < nfft):
                    continue
                for k in range(1, n + 1):
                    pts_j.append(int(OH.harmonic_row(jj, k, n, Z)))
                    pts_h.append(int(OH.harmonic_half_bin(hh, k, n)))
                    owners.append((ci, dj, dh))
    vals = oracle_plane_points(Ap, zmax, dz, extra, pts_j, pts_h)
    sums = {}
    for (ci, dj, dh), v in zip(owners, vals):
        sums[(ci, dj, dh)] = sums.get((ci, dj, dh), 0.0) + float(v)
    for ci, r in enumerate(rows):
        n, h, j = int(r["numharm"]), int(r["h"]), int(r["j"])
        s = sums[(ci, 0, 0)]
        assert abs(float(r["power"]) - s) <= P_RTOL * (s + n), (dm_idx, n, h, j, float(r["power"]), s)
        assert s >= thr[n] or abs(OST.sigma_of(n, s) - sigma_thr) < SIGMA_BAND, (dm_idx, n, h, j, s, thr[n])
        assert h >= OH.min_half_bin(n, t_span, f_lo), (dm_idx, n, h)
        for dj in (-1, 0, 1):
            for dh in (-1, 0, 1):
                key = (ci, dj, dh)
                if (dj, dh) == (0, 0) or key not in sums:
                    continue
                nb = sums[key]
                lin_me, lin_nb = j * nfft + h, (j + dj) * nfft + h + dh
                wins = s > nb or (s == nb and lin_me < lin_nb)
                assert wins or abs(nb - s) <= TIE_RTOL * s, (dm_idx, n, h, j, dj, dh, s, nb)
    return len(rows)
