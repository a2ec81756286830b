"""Candidate refinement objective in continuous (DM, r, z), FP64.

The paper folds candidates with prepfold (Sect. 2 step 6) to confirm them;
it does not refine (DM, period, acceleration) continuously.  This objective
is this project's definition (a reading), written from the shift theorem and
the drifting-sinusoid response of the acceleration search:

* Channel c's own spectrum A^c: its samples x_c[t] boxcar-downsampled by the
  trial's ds over the trial's valid length N_v (window starting at t = 0),
  minus their mean, zero-padded to nfft, transformed and truncated to nfft/2
  bins like the search's spectra.
* A continuous delay tau_c(DM) = K DM (f_c^-2 - f_ref^-2) seconds is undone by
  the phase exp(+i 2 pi f tau_c) at frequency f = k r / T (T = nfft ds tsamp).
* Harmonic k of the fundamental (r, z) sits at (k r, k z); its amplitude is
      F_k = sum_c exp(i phi_{c,k}) sum_{q=floor(kr)-m+1}^{floor(kr)+m} A^c_q conj(rho(kr - q, kz)),
  phi_{c,k} = 2 pi (k r) tau_c / T, m = m(kz) as for the plane, bins outside
  [0, nfft/2) contributing 0.
* P_h(DM, r, z) = sum_{k=1..h} g(floor(kr)) |F_k|^2 / E(kr, kz), where E is
  the template energy of those taps and g(bin) = ln 2 / med_b is the
  whitening gain of the block holding the bin, taken from the candidate's
  own DM trial (so P_h is close to S_h near a detection).
"""
from __future__ import annotations

import math

import numpy as np

from . import dedisperse as _dd
from . import plan as _plan
from . import response as _resp
from . import spectrum as _sp


def channel_spectra(x_cm: np.ndarray, nv: int, nfft: int, ds: int) -> np.ndarray:
    """complex128 [C][nfft/2]: per-channel mean-subtracted, padded spectra."""
    C = x_cm.shape[0]
    out = np.empty((C, nfft // 2), dtype=np.complex128)
    for c in range(C):
        s = x_cm[c, : nv * ds].astype(np.int64).reshape(nv, ds).sum(axis=1)
        out[c] = _sp.half_spectrum(_sp.real_series(s, nfft))
    return out


def whitening_gains(A: np.ndarray, block: int) -> np.ndarray:
    """ln 2 / med_b for each whitening block of a (raw) half spectrum, with
    the same block rules as spectrum.whiten (DC excluded; 0 if med is 0)."""
    M = A.shape[0]
    g = np.zeros(M // block)
    A = np.array(A, copy=True)
    A[0] = 0.0
    for b in range(M // block):
        p = np.abs(A[b * block:(b + 1) * block]) ** 2
        if b == 0:
            p = p[1:]
        med = _sp.lower_median(p)
        g[b] = math.log(2.0) / med if med > 0 else 0.0
    return g


class Objective:
    """P_h(DM, r, z) for one file, one DM trial's stage and its gains."""

    def __init__(self, fil, stages, cfg, dm_idx: int):
        self.P = _plan.Plan.for_file(fil, stages)
        self.x = _dd.channel_major(fil.data, fil.nchan, fil.nbits)
        self.dm_idx = int(dm_idx)
        self.ds = int(self.P.ds_of[dm_idx])
        self.nv, self.nfft = self.P.nv_nfft(dm_idx)
        self.T = self.P.t_span(dm_idx)
        self.cfg = cfg
        self.Ac = channel_spectra(self.x, self.nv, self.nfft, self.ds)
        s = _dd.dedisperse(self.x, self.P.delays[dm_idx], self.P.max_delay, self.ds)
        A = _sp.half_spectrum(_sp.real_series(s, self.nfft))
        self.gain = whitening_gains(A, cfg.whiten_block)
        f = self.P.freqs
        self.dtau = _plan.K_DM * (1.0 / (f * f) - 1.0 / (f.max() * f.max()))  # s per unit DM

    def harmonic(self, dm: float, r: float, z: float, k: int) -> float:
        M = self.nfft // 2
        rk, zk = k * r, k * z
        m = _resp.halfwidth(zk, self.cfg.halfwidth_extra)
        k0 = int(math.floor(rk))
        qs = np.arange(k0 - m + 1, k0 + m + 1)
        rho = np.array([_resp.rho(rk - q, zk) for q in qs])
        E = float(np.sum(np.abs(rho) ** 2))
        ok = (qs >= 0) & (qs < M)
        G = self.Ac[:, qs[ok]] @ np.conj(rho[ok])          # [C]
        phi = 2.0 * math.pi * rk * (dm * self.dtau) / self.T  # [C]
        F = np.sum(np.exp(1j * phi) * G)
        blk = min(max(k0, 0) // self.cfg.whiten_block, self.gain.shape[0] - 1)
        return float(self.gain[blk] * abs(F) ** 2 / E)

    def __call__(self, dm: float, r: float, z: float, numharm: int) -> float:
        return sum(self.harmonic(dm, r, z, k) for k in range(1, numharm + 1))

    def grid_max(self, dm0: float, r0: float, z0: float, numharm: int, dm_cell: float, dz: float):
        """Maximum over a fine grid of +-1 cell: DM in steps of dm_cell/8,
        r in steps of 1/16 bin, z in steps of dz/8 (z fixed when dz == 0)."""
        best = (-1.0, dm0, r0, z0)
        dms = dm0 + dm_cell / 8.0 * np.arange(-8, 9)
        rs = r0 + np.arange(-16, 17) / 16.0
        zs = [z0] if dz == 0 else z0 + dz / 8.0 * np.arange(-8, 9)
        for dm in dms:
            for r in rs:
                for z in zs:
                    v = self(float(dm), float(r), float(z), numharm)
                    if v > best[0]:
                        best = (v, float(dm), float(r), float(z))
        return best
