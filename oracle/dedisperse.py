"""Incoherent (shift-and-sum) dedispersion, exact in integers.

The paper dedisperses one DM per prepdata process (Sect. 2 step 2; Sect. 5
"Using other routines").  The operation is the textbook one: shift every
channel by its dispersion delay and sum over channels.
"""
from __future__ import annotations

import numpy as np


def channel_major(data: np.ndarray, nchan: int, nbits: int) -> np.ndarray:
    """uint8 [nchan][nsamp] from file-order (time-major) samples.

    8-bit: data is [nsamp][nchan].  1-bit: data is [nsamp][nchan/8] and
    channel c is bit (7 - c % 8) of byte c // 8 (reading: most significant
    bit first), value 0 or 1."""
    if nbits == 8:
        return np.ascontiguousarray(np.asarray(data, dtype=np.uint8)[:, :nchan].T)
    if nbits == 1:
        nsamp = data.shape[0]
        out = np.empty((nchan, nsamp), dtype=np.uint8)
        for c in range(nchan):
            out[c] = (data[:, c // 8] >> (7 - (c % 8))) & 1
        return out
    raise ValueError("nbits must be 8 or 1")


def dedisperse(x_cm: np.ndarray, delays_row: np.ndarray, max_delay: int, ds: int,
               chan_mask=None) -> np.ndarray:
    """int64 [N_v]: s[t] = sum_{c kept} x[c][t + d_c] for t < N - D, then
    boxcar downsampling s_ds[j] = sum_{k<ds} s[j*ds + k] for j < N_v.

    Reading: one valid length N - D (D = largest delay of the whole plan)
    for every trial; delays stay in native samples so the result is exact
    and independent of summation order."""
    nchan, nsamp = x_cm.shape
    L = nsamp - int(max_delay)
    s = np.zeros(L, dtype=np.int64)
    for c in range(nchan):
        if chan_mask is not None and not chan_mask[c]:
            continue
        d = int(delays_row[c])
        s += x_cm[c, d:d + L].astype(np.int64)
    nv = L // ds
    return s[: nv * ds].reshape(nv, ds).sum(axis=1)
