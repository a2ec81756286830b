"""Seeded synthetic filterbanks shaped like the paper's test data.

This module only *makes inputs*.  It holds none of the search's arithmetic
(no delay table, no dedispersion, no spectra): it simulates a radio
telescope's channelised, quantised output with periodic pulse trains whose
arrival time in each channel is shifted by the cold-plasma dispersion law,
evaluated here as a continuous time shift of the injected signal.

Shapes follow the paper's test files (Table 1: a 96-channel 1-bit PMPS file
of ~2100 s and a 200-channel 8-bit FAST file of 2^18 x 0.2 ms) and the
drift-scan file it sizes in Sect. 1 (256 channels, 0.2 ms, 8-bit, ~60 MB).
Real survey data is not available here; these files stand in for it.

Every array is produced from ``numpy.random.default_rng(seed)`` (PCG64), so
the same seed yields the same bytes on every machine that runs numpy >= 1.17.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Dispersion constant used to *simulate* the sky signal, s MHz^2 pc^-1 cm^3.
K_DISP_SIM = 4.148808e3
# Speed of light for converting a line-of-sight acceleration to a drift, m/s.
C_LIGHT = 299792458.0


@dataclasses.dataclass
class Pulsar:
    """One injected periodic source.

    period_s: barycentric period at t=0; dm: dispersion measure (pc cm^-3);
    duty: FWHM of the Gaussian pulse as a fraction of the period;
    amp: on-pulse peak amplitude per sample per channel in units of the
    noise standard deviation (8-bit) or the added on-pulse probability
    (1-bit); accel: constant line-of-sight acceleration in m/s^2;
    z_direct: if set, the total frequency drift over the file in Fourier
    bins of the fundamental (overrides accel); phase0: pulse phase at t=0.
    """

    period_s: float
    dm: float
    duty: float
    amp: float
    accel: float = 0.0
    z_direct: Optional[float] = None
    phase0: float = 0.0


@dataclasses.dataclass
class Filterbank:
    """A search-mode file held in memory.

    data is time-major (file order): uint8 [nsamp][nchan] for nbits=8, or
    uint8 [nsamp][nchan/8] for nbits=1 with channel c at bit (7 - c%8) of
    byte c//8 (most significant bit first).  fch0_mhz is the centre
    frequency of channel 0 and foff_mhz the signed channel spacing.
    """

    nchan: int
    nsamp: int
    tsamp_s: float
    fch0_mhz: float
    foff_mhz: float
    nbits: int
    data: np.ndarray
    pulsars: List[Pulsar]
    rfi_chans: Tuple[int, ...] = ()
    burst_t_s: Optional[float] = None

    def freqs_mhz(self) -> np.ndarray:
        return self.fch0_mhz + np.arange(self.nchan) * self.foff_mhz

    def nbytes(self) -> int:
        return int(self.data.size)


@dataclasses.dataclass
class Stage:
    """One dedispersion-plan row: n_dm trials DM_i = dm_lo + i*dm_step,
    time series downsampled by ds (the columns of the paper's Tables 2-3)."""

    dm_lo: float
    dm_step: float
    n_dm: int
    ds: int


@dataclasses.dataclass
class SearchCfg:
    zmax: int = 0
    dz: float = 2.0
    numharm: int = 8
    sigma_thr: float = 6.0
    f_lo_hz: float = 1.0
    whiten_block: int = 1024
    halfwidth_extra: int = 16
    min_dm_hits: int = 1


@dataclasses.dataclass
class Workload:
    name: str
    fil: Filterbank
    stages: List[Stage]
    cfg: SearchCfg


def band(lo_mhz: float, hi_mhz: float, nchan: int) -> Tuple[float, float]:
    """Channel-0 centre and spacing for nchan channels tiling [lo, hi] in
    ascending order."""
    foff = (hi_mhz - lo_mhz) / nchan
    return lo_mhz + 0.5 * foff, foff


def stages_from_table(rows: Sequence[Tuple[float, float, float, int]],
                      last_inclusive: bool) -> List[Stage]:
    """Build plan rows from (start, end, step, ds) as printed in a plan
    table.  Rows are half-open [start, end); if last_inclusive the final
    row also includes its end value (as in "DM 0-100 step 1, 101 trials")."""
    out = []
    for i, (lo, hi, step, ds) in enumerate(rows):
        n = int(round((hi - lo) / step))
        if last_inclusive and i == len(rows) - 1:
            n += 1
        out.append(Stage(float(lo), float(step), n, int(ds)))
    return out


def _gauss_profile(phase: np.ndarray, duty: float) -> np.ndarray:
    sig = duty / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    d = phase - np.floor(phase + 0.5)  # wrapped to [-0.5, 0.5)
    return np.exp(-0.5 * (d / sig) ** 2)


def _pulse_phase(p: Pulsar, t: np.ndarray, t_span: float) -> np.ndarray:
    """Rotational phase at emission time t (seconds) for a constant drift.

    With a constant frequency derivative fdot the phase is
    f0*t + fdot*t^2/2.  A line-of-sight acceleration a gives
    fdot = -f0*a/c; z_direct instead fixes fdot*T^2 = z (drift in bins)."""
    f0 = 1.0 / p.period_s
    if p.z_direct is not None:
        fdot = p.z_direct / (t_span * t_span)
    else:
        fdot = -f0 * p.accel / C_LIGHT
    return p.phase0 + f0 * t + 0.5 * fdot * t * t


def _sim_delay_s(dm: float, f_mhz: np.ndarray, f_top: float) -> np.ndarray:
    return K_DISP_SIM * dm * (1.0 / (f_mhz * f_mhz) - 1.0 / (f_top * f_top))


def _inject(x: np.ndarray, i0: int, tsamp: float, p: Pulsar, dly: np.ndarray, t_span: float,
            scale: float) -> None:
    """Add scale * profile of pulsar p to x[i][c] for samples i0 .. i0+len(x).

    The profile is exp(-d^2 / (2 s^2)), d the signed distance of the pulse
    phase to the nearest integer.  Without acceleration, pulse n arrives at
    t_n = (n - phase0) P + delay, and only samples within six profile widths
    (6 s in phase) of a pulse are touched (the profile is below 2e-8
    beyond); otherwise every sample is."""
    n = x.shape[0]
    sig = p.duty / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    nchan = x.shape[1]
    if p.accel == 0.0 and p.z_direct is None and 6.0 * sig < 0.5:
        f0 = 1.0 / p.period_s
        w = int(math.ceil(6.0 * sig * p.period_s / tsamp)) + 1
        offs = np.arange(-w, w + 1)
        for c in range(nchan):
            t_lo = i0 * tsamp - dly[c]
            t_hi = (i0 + n) * tsamp - dly[c]
            k_lo = int(math.floor(p.phase0 + f0 * t_lo)) - 1
            k_hi = int(math.ceil(p.phase0 + f0 * t_hi)) + 1
            ks = np.arange(k_lo, k_hi + 1)
            tn = (ks - p.phase0) / f0 + dly[c]                  # arrival times
            idx = np.rint(tn / tsamp).astype(np.int64)[:, None] + offs[None, :]
            ok = (idx >= i0) & (idx < i0 + n)
            ii = idx[ok]
            kk = np.broadcast_to(ks[:, None], idx.shape)[ok]
            d = (p.phase0 + f0 * (ii * tsamp - dly[c])) - kk
            np.add.at(x[:, c], ii - i0, scale * np.exp(-0.5 * (d / sig) ** 2))
        return
    t = np.arange(i0, i0 + n, dtype=np.float64) * tsamp
    for c in range(nchan):
        x[:, c] += scale * _gauss_profile(_pulse_phase(p, t - dly[c], t_span), p.duty)


def make_8bit(nchan: int, nsamp: int, tsamp: float, lo: float, hi: float,
              pulsars: Sequence[Pulsar], seed: int,
              rfi_chans: Sequence[int] = (), burst_t_s: Optional[float] = None,
              ) -> Filterbank:
    """uint8 noise clip(round_half_even(128 + 16 g), 0, 255), g ~ N(0,1),
    plus dispersed pulses (amplitude in noise sd), narrowband RFI (a 50 Hz
    sinusoid of 3 sd in each listed channel) and a zero-DM burst (+4 sd in
    every channel for 5 ms), all added before quantisation."""
    rng = np.random.default_rng(seed)
    fch0, foff = band(lo, hi, nchan)
    freqs = fch0 + np.arange(nchan) * foff
    f_top = float(freqs.max())
    t = np.arange(nsamp, dtype=np.float64) * tsamp
    t_span = nsamp * tsamp
    x = np.empty((nsamp, nchan), dtype=np.float64)
    for c0 in range(0, nchan, 32):
        c1 = min(nchan, c0 + 32)
        x[:, c0:c1] = rng.standard_normal((nsamp, c1 - c0))
    for p in pulsars:
        _inject(x, 0, tsamp, p, _sim_delay_s(p.dm, freqs, f_top), t_span, p.amp)
    for c in rfi_chans:
        x[:, c] += 3.0 * np.sin(2.0 * math.pi * 50.0 * t)
    if burst_t_s is not None:
        i0 = int(burst_t_s / tsamp)
        i1 = min(nsamp, i0 + max(1, int(5e-3 / tsamp)))
        x[i0:i1, :] += 4.0
    q = np.clip(np.rint(128.0 + 16.0 * x), 0, 255).astype(np.uint8)
    return Filterbank(nchan, nsamp, tsamp, fch0, foff, 8, np.ascontiguousarray(q),
                      list(pulsars), tuple(rfi_chans), burst_t_s)


_QTAB = None


def _quantised_gauss_table() -> np.ndarray:
    """uint8 [65536]: a uniform 16-bit index maps to clip(round(128 + 16 g),
    0, 255) with the probabilities of g ~ N(0, 1) (to 2^-16)."""
    global _QTAB
    if _QTAB is None:
        v = np.arange(256)
        edges = (v[:-1] + 0.5 - 128.0) / 16.0                  # upper edge of each value
        cdf = 0.5 * (1.0 + np.array([math.erf(e / math.sqrt(2.0)) for e in edges]))
        cut = np.rint(cdf * 65536.0).astype(np.int64)          # first index of value v+1
        tab = np.searchsorted(cut, np.arange(65536), side="right").astype(np.uint8)
        _QTAB = tab
    return _QTAB


def make_8bit_stream(nchan: int, nsamp: int, tsamp: float, lo: float, hi: float,
                     pulsars: Sequence[Pulsar], seed: int) -> Filterbank:
    """A fast stand-in for make_8bit for the many large files of a served
    stream: the noise values are drawn directly with the distribution of the
    quantised Gaussian (a 16-bit lookup table), and each pulsar's pulse train
    (Gaussian profile, FWHM duty * P) is added in the quantised domain
    (stochastically rounded to 1/16 sd, so its mean is kept) at the channel's
    dispersion delay rounded to a whole sample."""
    rng = np.random.default_rng(seed)
    fch0, foff = band(lo, hi, nchan)
    freqs = fch0 + np.arange(nchan) * foff
    f_top = float(freqs.max())
    q = _quantised_gauss_table()[rng.integers(0, 65536, (nsamp, nchan), dtype=np.uint16)]
    t = np.arange(nsamp, dtype=np.float64) * tsamp
    for p in pulsars:
        ph = p.phase0 + t / p.period_s
        v = 16.0 * p.amp * _gauss_profile(ph, p.duty)
        nz = np.nonzero(v > 1e-3)[0]
        if nz.size == 0:
            continue
        sh = np.rint(_sim_delay_s(p.dm, freqs, f_top) / tsamp).astype(np.int64)
        for c in range(nchan):
            idx = nz + sh[c]
            keep = idx < nsamp
            # stochastic rounding keeps the mean of a sub-level pulse
            inc = np.floor(v[nz[keep]] + rng.random(int(keep.sum()))).astype(np.int16)
            col = q[idx[keep], c].astype(np.int16) + inc
            q[idx[keep], c] = np.clip(col, 0, 255).astype(np.uint8)
    return Filterbank(nchan, nsamp, tsamp, fch0, foff, 8, q, list(pulsars))


def make_1bit(nchan: int, nsamp: int, tsamp: float, lo: float, hi: float,
              pulsars: Sequence[Pulsar], seed: int, chunk: int = 1 << 18,
              ) -> Filterbank:
    """Bernoulli(0.5) bits; on-pulse the probability is raised by
    amp*profile.  Packed MSB-first, 8 channels per byte, time-major."""
    assert nchan % 8 == 0
    rng = np.random.default_rng(seed)
    fch0, foff = band(lo, hi, nchan)
    freqs = fch0 + np.arange(nchan) * foff
    f_top = float(freqs.max())
    t_span = nsamp * tsamp
    out = np.empty((nsamp, nchan // 8), dtype=np.uint8)
    for s0 in range(0, nsamp, chunk):
        s1 = min(nsamp, s0 + chunk)
        u = rng.random((s1 - s0, nchan))
        prob = np.full((s1 - s0, nchan), 0.5)
        for p in pulsars:
            _inject(prob, s0, tsamp, p, _sim_delay_s(p.dm, freqs, f_top), t_span, p.amp)
        bits = (u < prob).astype(np.uint8)
        out[s0:s1] = np.packbits(bits, axis=1, bitorder="big")
    return Filterbank(nchan, nsamp, tsamp, fch0, foff, 1, out, list(pulsars))


def unpack_bits(fil: Filterbank) -> np.ndarray:
    """Time-major uint8 [nsamp][nchan] of 0/1 values from a 1-bit file."""
    return np.unpackbits(fil.data, axis=1, bitorder="big")[:, : fil.nchan]


# ---------------------------------------------------------------------------
# Workloads shaped like the paper's data (Sect. 1; Table 1; Tables 2-3).
# ---------------------------------------------------------------------------

def workload_small(seed: int = 1001, nsamp: int = 1 << 16) -> Workload:
    """64 channels over 1200-1500 MHz, 0.2 ms, 2^16 samples, one pulsar
    (P = 33.3 ms, DM 50, 5 % duty, 0.5 sd); DM 0-100 step 1 (101 trials),
    zmax 0, harmonic sums up to 8, 6 sigma."""
    fil = make_8bit(64, nsamp, 2e-4, 1200.0, 1500.0,
                    [Pulsar(0.0333, 50.0, 0.05, 0.5, phase0=0.1)], seed)
    return Workload("small_64ch_2^16_zmax0", fil, [Stage(0.0, 1.0, 101, 1)],
                    SearchCfg(zmax=0, numharm=8))


def _drift_pulsars(rng: np.random.Generator, n: int, nchan: int, nsamp: int) -> List[Pulsar]:
    out = []
    for _ in range(n):
        P = rng.uniform(0.002, 0.5)
        dm = rng.uniform(10.0, 500.0)
        duty = rng.uniform(0.02, 0.10)
        target = rng.uniform(8.0, 30.0)
        amp = target / math.sqrt(nchan * nsamp * duty)
        out.append(Pulsar(P, dm, duty, amp, phase0=rng.uniform()))
    return out


def workload_driftscan(seed: int = 1002, nsamp: int = 1 << 18, nchan: int = 256,
                       n_dm: int = 1001) -> Workload:
    """256 channels over 1050-1450 MHz, 0.2 ms, 2^18 samples (52.4 s), five
    pulsars (P 2-500 ms, DM 10-500, duty 2-10 %, 8-30 sigma folded), three
    narrowband RFI channels and one zero-DM burst; DM 0-500 step 0.5
    (1001 trials), zmax 0, harmonic sums up to 16."""
    rng = np.random.default_rng(seed + 7)
    psrs = _drift_pulsars(rng, 5, nchan, nsamp)
    rfi = tuple(int(c) for c in rng.choice(nchan, 3, replace=False))
    fil = make_8bit(nchan, nsamp, 2e-4, 1050.0, 1450.0, psrs, seed,
                    rfi_chans=rfi, burst_t_s=0.37 * nsamp * 2e-4)
    return Workload("driftscan_256ch_2^18_zmax0", fil, [Stage(0.0, 0.5, n_dm, 1)],
                    SearchCfg(zmax=0, numharm=16))


def workload_accel(seed: int = 1003, nsamp: int = 1 << 18, nchan: int = 256,
                   n_dm: int = 301, zmax: int = 200) -> Workload:
    """The drift-scan file shape with three binary pulsars (P 2-50 ms,
    line-of-sight acceleration 1-50 m/s^2, DM 20-300) plus two pulsars
    whose drift is given directly in bins (z = +37 and -151) so that
    |z| > 0 cells of the f-fdot plane are exercised; DM 0-300 step 1,
    zmax 200, dz 2, harmonic sums up to 8."""
    rng = np.random.default_rng(seed + 7)
    psrs = []
    for _ in range(3):
        P = rng.uniform(0.002, 0.05)
        psrs.append(Pulsar(P, rng.uniform(20.0, 300.0), rng.uniform(0.03, 0.08),
                           rng.uniform(0.08, 0.15), accel=rng.uniform(1.0, 50.0),
                           phase0=rng.uniform()))
    for z in (37.0, -151.0):
        psrs.append(Pulsar(rng.uniform(0.004, 0.02), rng.uniform(20.0, 300.0), 0.05,
                           0.15, z_direct=z, phase0=rng.uniform()))
    fil = make_8bit(nchan, nsamp, 2e-4, 1050.0, 1450.0, psrs, seed)
    return Workload("accel_256ch_2^18_zmax%d" % zmax, fil, [Stage(0.0, 1.0, n_dm, 1)],
                    SearchCfg(zmax=zmax, dz=2.0, numharm=8))


def workload_pmps(seed: int = 1004, nsamp: int = 1 << 23, zmax: int = 0,
                  scale_dm: float = 1.0) -> Workload:
    """96 channels over 1230-1518 MHz (3 MHz), 0.25 ms, 2^23 samples,
    1-bit; three pulsars raising the on-pulse probability by 0.02-0.1;
    staged plan 0-200 step 0.5, 200-600 step 1 (ds 2), 600-2000 step 5
    (ds 4, end inclusive); harmonic sums up to 16."""
    rng = np.random.default_rng(seed + 7)
    psrs = [Pulsar(rng.uniform(0.005, 0.5), rng.uniform(20.0, 1500.0) * scale_dm,
                   rng.uniform(0.03, 0.08), rng.uniform(0.02, 0.1), phase0=rng.uniform())
            for _ in range(3)]
    fil = make_1bit(96, nsamp, 2.5e-4, 1230.0, 1518.0, psrs, seed)
    rows = [(0.0, 200.0, 0.5, 1), (200.0, 600.0, 1.0, 2), (600.0, 2000.0, 5.0, 4)]
    return Workload("pmps_96ch_1bit_2^23_zmax%d" % zmax, fil,
                    stages_from_table(rows, last_inclusive=True),
                    SearchCfg(zmax=zmax, dz=2.0, numharm=16))


# The paper's FAST drift-scan plan (Table 3): rows (start, end, step, ds),
# each row the half-open range [start, end); 979 trials in all.
TABLE3_ROWS = ((0.0, 31.5, 0.1, 8), (31.5, 62.9, 0.2, 16), (62.9, 139.4, 0.5, 32),
               (139.4, 278.4, 1.0, 64), (278.4, 556.4, 2.0, 128), (556.4, 784.4, 3.0, 128))


def workload_fast(seed: int = 1006, nsamp: int = 1 << 18, zmax: int = 0) -> Workload:
    """The paper's FAST test file shape (Table 1; timed in Sect. 3.3): 200 channels
    over 290-340 MHz, 0.2 ms, 2^18 samples, 8-bit, searched with the
    Table 3 plan (979 trials, ds 8-128).  Five pulsars (P 0.1-0.9 s, so
    that the channel smearing at these frequencies, tens of ms at the
    highest DMs, stays below a tenth of the period; DM 10-700; duty 2-8 %;
    8-30 sigma folded), two narrowband RFI channels and a zero-DM burst;
    harmonic sums up to 16."""
    nchan = 200
    rng = np.random.default_rng(seed + 7)
    psrs = []
    for _ in range(5):
        duty = rng.uniform(0.02, 0.08)
        amp = rng.uniform(8.0, 30.0) / math.sqrt(nchan * nsamp * duty)
        psrs.append(Pulsar(rng.uniform(0.1, 0.9), rng.uniform(10.0, 700.0), duty, amp, phase0=rng.uniform()))
    rfi = tuple(int(c) for c in rng.choice(nchan, 2, replace=False))
    fil = make_8bit(nchan, nsamp, 2e-4, 290.0, 340.0, psrs, seed, rfi_chans=rfi,
                    burst_t_s=0.61 * nsamp * 2e-4)
    return Workload("fast_200ch_2^18_table3_zmax%d" % zmax, fil,
                    stages_from_table(TABLE3_ROWS, last_inclusive=False),
                    SearchCfg(zmax=zmax, dz=2.0, numharm=16))


def stream_files(n_files: int = 64, seed0: int = 5000, mean_gap_s: float = 26.0,
                 speedup: float = 50.0, max_log2: int = 19, chans=(128, 256, 512, 1024)):
    """A drift-scan stream: n_files files with channel counts drawn from
    chans, 2^17..2^max_log2 samples, 0-3 pulsars each, arriving at Poisson
    intervals (mean 26 s, replayed faster by `speedup`).  Yields
    (arrival_s, Workload)."""
    rng = np.random.default_rng(seed0)
    t = 0.0
    for f in range(n_files):
        t += rng.exponential(mean_gap_s) / speedup
        nchan = int(rng.choice(chans))
        nsamp = 1 << int(rng.integers(17, max_log2 + 1))
        npsr = int(rng.integers(0, 4))
        prng = np.random.default_rng(seed0 + f + 100000)
        psrs = _drift_pulsars(prng, npsr, nchan, nsamp)
        fil = make_8bit_stream(nchan, nsamp, 2e-4, 1050.0, 1450.0, psrs, seed0 + f)
        yield t, Workload("stream_file_%d" % f, fil, [Stage(0.0, 1.0, 501, 1)],
                          SearchCfg(zmax=100, dz=2.0, numharm=8))
