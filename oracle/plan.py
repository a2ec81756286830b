"""Dedispersion plan: channel frequencies, DM grid, integer delay table.

The paper generates its DM plans with DDplan (Sect. 3.1, Tables 2 and 3:
start, end, step, downsample factor, number of DMs per row).  The delay
law itself is not written in the paper; the textbook cold-plasma delay
t(f) = K_DM * DM / f^2 is used, referenced to the highest channel.
"""
from __future__ import annotations

import numpy as np

# Dispersion constant in s MHz^2 pc^-1 cm^3 (the paper quotes none).
K_DM = 4.148808e3


def channel_freqs(nchan: int, fch0_mhz: float, foff_mhz: float) -> np.ndarray:
    """Centre frequency of each channel.  Reading: fch0 is the centre of
    channel 0, so f_c = fch0 + c*foff (FP64)."""
    return fch0_mhz + np.arange(nchan, dtype=np.float64) * foff_mhz


def dm_grid(stages):
    """All DM trials of a plan, stage by stage.

    Each stage (dm_lo, dm_step, n_dm, ds) contributes DM_i = dm_lo + i*dm_step
    for i < n_dm, each value computed directly in FP64 (no running sum), as
    the rows of Tables 2-3 list start, step and count.  Returns
    (dms float64 [ndm], stage_of int [ndm], ds_of int [ndm])."""
    dms, st, dss = [], [], []
    for s_idx, s in enumerate(stages):
        for i in range(int(s.n_dm)):
            dms.append(float(s.dm_lo) + float(i) * float(s.dm_step))
            st.append(s_idx)
            dss.append(int(s.ds))
    return np.array(dms, dtype=np.float64), np.array(st, dtype=np.int64), np.array(dss, dtype=np.int64)


def round_half_away(x: np.ndarray) -> np.ndarray:
    """Round to nearest integer, halves away from zero (C ``round``)."""
    x = np.asarray(x, dtype=np.float64)
    t = np.trunc(x)
    frac = x - t  # exact for |x| < 2^52
    return (t + np.sign(x) * (np.abs(frac) >= 0.5)).astype(np.int64)


def delay_values(dms: np.ndarray, freqs: np.ndarray, tsamp_s: float) -> np.ndarray:
    """Unrounded delays in samples, evaluated in FP64 in the fixed order
    ((K_DM*DM) * (1/(f_c*f_c) - 1/(f_ref*f_ref))) / tsamp.

    Reading: f_ref is the highest channel frequency, so every delay is >= 0."""
    freqs = np.asarray(freqs, dtype=np.float64)
    f_ref = float(freqs.max())
    inv_ref = 1.0 / (f_ref * f_ref)
    diff = 1.0 / (freqs * freqs) - inv_ref
    kd = K_DM * np.asarray(dms, dtype=np.float64)
    return (kd[:, None] * diff[None, :]) / tsamp_s


def delay_table(dms: np.ndarray, freqs: np.ndarray, tsamp_s: float) -> np.ndarray:
    """int64 [ndm][nchan] integer sample delays d_c(DM), rounded half away
    from zero."""
    return round_half_away(delay_values(dms, freqs, tsamp_s))


def next_pow2(n: int) -> int:
    p = 1
    while p < n:
        p <<= 1
    return p


def stage_lengths(nsamp: int, max_delay: int, ds: int):
    """(N_v, nfft) of one stage.  Reading: one valid length N - D for every
    trial (D = the largest delay in the whole plan), boxcar-downsampled by
    ds, zero-padded to the next power of two."""
    if nsamp <= max_delay:
        raise ValueError("file shorter than the largest dispersion delay")
    nv = (nsamp - max_delay) // ds
    if nv < 1:
        raise ValueError("no valid samples after downsampling")
    return nv, next_pow2(nv)


class Plan:
    """Everything the search needs from the plan, computed once.

    subband = (nsub, group) selects the two-stage scheme of
    `oracle.subband` (self.sub); its largest combined delay then also bounds
    the valid length (D' = max(D, that delay))."""

    def __init__(self, nchan, nsamp, tsamp_s, fch0_mhz, foff_mhz, stages, subband=None):
        self.nchan, self.nsamp, self.tsamp_s = int(nchan), int(nsamp), float(tsamp_s)
        self.freqs = channel_freqs(nchan, fch0_mhz, foff_mhz)
        self.stages = list(stages)
        self.dms, self.stage_of, self.ds_of = dm_grid(self.stages)
        self.delays = delay_table(self.dms, self.freqs, self.tsamp_s)
        self.max_delay = int(self.delays.max()) if self.delays.size else 0
        self.sub = None
        if subband is not None:
            from .subband import SubbandPlan
            self.sub = SubbandPlan(self.freqs, self.dms, self.stage_of, self.tsamp_s, *subband)
            self.max_delay = max(self.max_delay, self.sub.max_comb)
        self.lengths = [stage_lengths(self.nsamp, self.max_delay, int(s.ds)) for s in self.stages]

    @classmethod
    def for_file(cls, fil, stages, subband=None):
        return cls(fil.nchan, fil.nsamp, fil.tsamp_s, fil.fch0_mhz, fil.foff_mhz, stages, subband)

    def nv_nfft(self, dm_idx: int):
        return self.lengths[int(self.stage_of[dm_idx])]

    def t_span(self, dm_idx: int) -> float:
        """T = nfft * ds * tsamp, the span of the transformed series; Fourier
        bin r corresponds to r / T Hz."""
        _, nfft = self.nv_nfft(dm_idx)
        return float(nfft * int(self.ds_of[dm_idx])) * self.tsamp_s
