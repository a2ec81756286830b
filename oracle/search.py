"""The whole per-DM-trial search, step by step in the order of the paper's
pipeline (Sect. 2 steps 2-5): dedisperse -> FFT -> (acceleration) search
-> sift.  Each step is the function of the same name in this package.
"""
from __future__ import annotations

from typing import Dict, Iterable, List, Optional

import numpy as np

from . import dedisperse as _dd
from . import harmsum as _hs
from . import plan as _plan
from . import response as _resp
from . import sift as _sift
from . import spectrum as _sp
from . import subband as _sb
from . import stats as _st


def spectrum_of_trial(x_cm, P: _plan.Plan, dm_idx: int, block: int, chan_mask=None):
    """(s int64 [N_v], A' complex128 [nfft/2]) for one DM trial."""
    ds = int(P.ds_of[dm_idx])
    nv, nfft = P.nv_nfft(dm_idx)
    if P.sub is None:
        s = _dd.dedisperse(x_cm, P.delays[dm_idx], P.max_delay, ds, chan_mask)
    else:
        s = _sb.dedisperse_subband(x_cm, P.sub, dm_idx, P.max_delay, ds, chan_mask)
    assert s.shape[0] == nv
    y = _sp.real_series(s, nfft)
    A = _sp.half_spectrum(y)
    return s, _sp.whiten(A, block)


def search_trial(x_cm, P: _plan.Plan, dm_idx: int, cfg, thr: Optional[dict] = None,
                 plane_method: str = "direct", chan_mask=None) -> List[Dict]:
    """Raw candidates of one DM trial as dicts with dm_idx, numharm, h, j,
    power (S_n), sigma, r, z, f_hz."""
    if thr is None:
        thr = _st.thresholds(cfg.numharm, cfg.sigma_thr)
    _, Ap = spectrum_of_trial(x_cm, P, dm_idx, cfg.whiten_block, chan_mask)
    plane = _resp.power_plane(Ap, cfg.zmax, cfg.dz, cfg.halfwidth_extra, plane_method)
    Z = int(round(cfg.zmax / cfg.dz)) if cfg.zmax else 0
    T = P.t_span(dm_idx)
    out = []
    for n, h, j, S in _hs.raw_candidates(plane, cfg.numharm, Z, thr, T, cfg.f_lo_hz):
        r, z = _sift.fundamental(n, h, j, Z, cfg.dz)
        out.append(dict(dm_idx=int(dm_idx), dm=float(P.dms[dm_idx]), numharm=n, h=h, j=j,
                        power=S, sigma=_st.sigma_of(n, S), r=r, z=z, zq=_sift.zq(n, j, Z), f_hz=r / T))
    return out


def search(fil, stages, cfg, dm_indices: Optional[Iterable[int]] = None,
           plane_method: str = "direct", subband=None):
    """(raw candidates by DM index, sifted list) for a file; subband =
    (nsub, group) dedisperses by the two-stage scheme (oracle.subband)."""
    P = _plan.Plan.for_file(fil, stages, subband)
    x_cm = _dd.channel_major(fil.data, fil.nchan, fil.nbits)
    thr = _st.thresholds(cfg.numharm, cfg.sigma_thr)
    idx = range(len(P.dms)) if dm_indices is None else dm_indices
    raw = {int(i): search_trial(x_cm, P, int(i), cfg, thr, plane_method) for i in idx}
    return raw, _sift.sift(raw, cfg.dz, cfg.min_dm_hits)
