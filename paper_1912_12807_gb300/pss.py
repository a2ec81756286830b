"""ctypes binding of libpss (declared in include/pss.h).

Argument marshalling only: every step of the search runs in the CUDA
library.  Device buffers are torch tensors on the context's GPU; host
buffers are numpy arrays.  The functions keep the C names.  If the shared
library has not been built, importing this module raises -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpss.so")

PSS_OK, PSS_EINVAL, PSS_ENOMEM, PSS_ECAP, PSS_ETIMEOUT, PSS_ECUDA, PSS_EBUSY, PSS_ENOTREADY = 0, -1, -2, -3, -4, -5, -6, -7
_NAMES = {0: "PSS_OK", -1: "PSS_EINVAL", -2: "PSS_ENOMEM", -3: "PSS_ECAP", -4: "PSS_ETIMEOUT", -5: "PSS_ECUDA",
          -6: "PSS_EBUSY", -7: "PSS_ENOTREADY"}


class PssError(RuntimeError):
    def __init__(self, status: int, msg: str, needed: Optional[int] = None):
        super().__init__("%s: %s" % (_NAMES.get(status, status), msg))
        self.status = status
        self.needed = needed


class pss_fil_desc(C.Structure):
    _fields_ = [("nchan", C.c_int32), ("nbits", C.c_int32), ("nsamp", C.c_int64), ("tsamp_s", C.c_double),
                ("fch0_mhz", C.c_double), ("foff_mhz", C.c_double), ("layout", C.c_int32),
                ("reserved", C.c_int32), ("chan_mask", C.POINTER(C.c_uint8))]


class pss_dd_stage(C.Structure):
    _fields_ = [("dm_lo", C.c_double), ("dm_step", C.c_double), ("n_dm", C.c_int32), ("ds", C.c_int32)]


class pss_search_cfg(C.Structure):
    _fields_ = [("zmax", C.c_int32), ("numharm", C.c_int32), ("dz", C.c_double), ("sigma_thr", C.c_double),
                ("f_lo_hz", C.c_double), ("whiten_block", C.c_int32), ("halfwidth_extra", C.c_int32),
                ("min_dm_hits", C.c_int32), ("reserved", C.c_int32)]


class pss_refine_point(C.Structure):
    _fields_ = [("dm_idx", C.c_int32), ("numharm", C.c_int32), ("dm", C.c_double), ("r", C.c_double),
                ("z", C.c_double)]


REFINE_DTYPE = np.dtype([("dm_idx", "<i4"), ("numharm", "<i4"), ("dm", "<f8"), ("r", "<f8"), ("z", "<f8")])
RAW_DTYPE = np.dtype([("dm_idx", "<i4"), ("numharm", "<i4"), ("h", "<i4"), ("j", "<i4"), ("power", "<f4"),
                      ("reserved", "<i4")])
FOLD_REQ_DTYPE = np.dtype([("dm_idx", "<i4"), ("reserved", "<i4"), ("f_hz", "<f8"), ("fdot_hz_s", "<f8")])
FOLD_RES_DTYPE = np.dtype([("f_hz", "<f8"), ("chi2_red", "<f8"), ("best", "<i4"), ("reserved", "<i4")])
SP_DTYPE = np.dtype([("dm_idx", "<i4"), ("width", "<i4"), ("t", "<i8"), ("boxsum", "<i8"), ("snr", "<f8")])
SP_WIDTHS = (1, 2, 3, 4, 6, 9, 14, 20, 30, 45, 70, 100, 150)
CAND_DTYPE = np.dtype([("dm_idx", "<i4"), ("numharm", "<i4"), ("dm", "<f8"), ("r", "<f8"), ("z", "<f8"),
                       ("f_hz", "<f8"), ("sigma", "<f8"), ("power", "<f4"), ("dm_hits", "<i4"), ("h", "<i4"),
                       ("j", "<i4")], align=True)

# every symbol include/pss.h declares
EXPORTS = ["pss_ctx_create", "pss_ctx_destroy", "pss_last_error", "pss_version", "pss_dd_plan", "pss_dd_plan_auto", "pss_dd_plan_subband",
           "pss_plan_subband_info", "pss_plan_info",
           "pss_plan_trial_info", "pss_plan_free", "pss_dedisperse", "pss_single_pulse", "pss_fold", "pss_spectrum", "pss_power_plane",
           "pss_search_raw", "pss_sift", "pss_sift_in_batches", "pss_search_dm_batch", "pss_response", "pss_sigma_of_power",
           "pss_power_threshold", "pss_ctx_profile", "pss_ctx_profile_read", "pss_dedisperse_noalloc",
           "pss_refine_prepare", "pss_refine_eval", "pss_refine_candidates", "pss_batch_create", "pss_batch_run",
           "pss_batch_footprint", "pss_batch_free", "pss_search_footprint", "pss_ctx_take_cands",
           "pss_batch_take_cands", "pss_batch_tuning", "pss_batch_fft_split", "pss_fft_split_radices",
           "pss_ctx_set_fft_split", "pss_measure_peaks", "pss_ctx_set_wait_limit", "pss_debug_fail_alloc",
           "pss_ctx_check", "pss_search_multi", "pss_search_multi_footprint",
           "pss_server_create", "pss_server_create_grouped", "pss_server_group_stats", "pss_submit_file",
           "pss_submit_file_subband", "pss_poll",
           "pss_result_cands", "pss_result_free", "pss_server_stats", "pss_server_destroy"]
PROFILE_STAGES = ["unpack", "dedisperse", "fft", "whiten", "plane", "harmsum", "bxtable"]

_lib = None


def lib():
    """The loaded libpss (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libpss.so not built (run python -m paper_1912_12807_gb300.build): " + LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, st = C.c_void_p, C.c_int64, C.c_int32, C.c_int
    P = C.POINTER
    sig = {
        "pss_ctx_create": (st, [C.c_int, P(vp)]),
        "pss_ctx_destroy": (None, [vp]),
        "pss_last_error": (C.c_char_p, []),
        "pss_version": (C.c_char_p, []),
        "pss_dd_plan": (st, [P(pss_fil_desc), P(pss_dd_stage), C.c_int, P(vp)]),
        "pss_dd_plan_auto": (st, [P(pss_fil_desc), C.c_double, C.c_double, C.c_double, i32, vp, i32, P(i32)]),
        "pss_dd_plan_subband": (st, [P(pss_fil_desc), P(pss_dd_stage), C.c_int, i32, i32, P(vp)]),
        "pss_plan_subband_info": (st, [vp, P(i32), P(i32), P(i64), vp, vp, vp]),
        "pss_plan_info": (st, [vp, P(i64), P(i64), vp, vp]),
        "pss_plan_trial_info": (st, [vp, i64, P(i32), P(i64), P(i64), P(i32)]),
        "pss_plan_free": (None, [vp]),
        "pss_dedisperse": (st, [vp, vp, P(pss_fil_desc), vp, C.c_int, i64, i64, vp, vp]),
        "pss_single_pulse": (st, [vp, vp, P(pss_fil_desc), vp, C.c_int, i64, i64, vp, i32, C.c_double, vp, i64,
                                  P(i64), vp]),
        "pss_fold": (st, [vp, vp, P(pss_fil_desc), vp, C.c_int, vp, i64, i32, i32, C.c_double, vp, vp, vp, vp]),
        "pss_spectrum": (st, [vp, vp, P(pss_fil_desc), vp, C.c_int, P(pss_search_cfg), i64, i64, vp, vp]),
        "pss_power_plane": (st, [vp, vp, P(pss_fil_desc), vp, C.c_int, P(pss_search_cfg), i64, i64, vp, vp]),
        "pss_search_raw": (st, [vp, vp, P(pss_fil_desc), vp, C.c_int, P(pss_search_cfg), i64, i64, vp, i64,
                                P(i64), vp]),
        "pss_sift": (st, [vp, P(pss_search_cfg), vp, i64, vp, i64, P(i64)]),
        "pss_sift_in_batches": (st, [vp, P(pss_search_cfg), vp, i64, vp, i32, vp, i64, P(i64)]),
        "pss_search_dm_batch": (st, [vp, vp, P(pss_fil_desc), vp, C.c_int, P(pss_search_cfg), i64, i64, vp, i64,
                                     P(i64), vp]),
        "pss_response": (st, [vp, vp, vp, i64, vp]),
        "pss_dedisperse_noalloc": (st, [vp, P(pss_fil_desc), vp, i64, i64, vp, vp]),
        "pss_refine_prepare": (st, [vp, vp, P(pss_fil_desc), vp, C.c_int, P(pss_search_cfg), i32, vp]),
        "pss_refine_eval": (st, [vp, vp, vp, i64, vp, vp, vp]),
        "pss_refine_candidates": (st, [vp, vp, P(pss_fil_desc), vp, C.c_int, P(pss_search_cfg), vp, i64, i32,
                                       C.c_double, vp]),
        "pss_ctx_profile": (st, [vp, C.c_int]),
        "pss_ctx_profile_read": (st, [vp, vp, vp]),
        "pss_batch_create": (st, [C.c_int, vp, P(pss_fil_desc), P(pss_search_cfg), P(vp)]),
        "pss_batch_run": (st, [vp, vp, C.c_int, vp, i64, P(i64), P(C.c_double)]),
        "pss_batch_footprint": (C.c_size_t, [vp]),
        "pss_batch_free": (None, [vp]),
        "pss_ctx_take_cands": (st, [vp, vp, i64, P(i64)]),
        "pss_batch_take_cands": (st, [vp, vp, i64, P(i64)]),
        "pss_batch_tuning": (st, [vp, P(i32), P(i32), P(i32), P(i32), P(i32)]),
        "pss_batch_fft_split": (st, [vp, i64, P(i32)]),
        "pss_fft_split_radices": (st, [i64, i32, P(i32), P(i32)]),
        "pss_ctx_set_fft_split": (st, [vp, i64, i32]),
        "pss_measure_peaks": (st, [C.c_int, vp]),
        "pss_ctx_set_wait_limit": (st, [vp, i32]),
        "pss_ctx_check": (st, [vp, vp]),
        "pss_debug_fail_alloc": (None, [i64]),
        "pss_search_multi": (st, [vp, P(pss_search_cfg), vp, i32, C.c_int, vp, i64, vp, P(i64), vp]),
        "pss_search_multi_footprint": (st, [P(pss_search_cfg), vp, i32, P(C.c_size_t)]),
        "pss_search_footprint": (st, [vp, P(pss_fil_desc), P(pss_search_cfg), P(C.c_size_t)]),
        "pss_server_create": (st, [C.c_int, C.c_size_t, C.c_int, P(vp)]),
        "pss_server_create_grouped": (st, [C.c_int, C.c_size_t, C.c_int, C.c_int, P(vp)]),
        "pss_server_group_stats": (st, [vp, P(i64), P(i64)]),
        "pss_submit_file": (st, [vp, P(pss_fil_desc), vp, P(pss_dd_stage), C.c_int, P(pss_search_cfg),
                                 P(C.c_uint64)]),
        "pss_submit_file_subband": (st, [vp, P(pss_fil_desc), vp, P(pss_dd_stage), C.c_int, i32, i32,
                                         P(pss_search_cfg), P(C.c_uint64)]),
        "pss_poll": (st, [vp, C.c_uint64, C.c_int, P(vp)]),
        "pss_result_cands": (st, [vp, P(vp), P(i64), P(C.c_double)]),
        "pss_result_free": (None, [vp]),
        "pss_server_stats": (st, [vp, P(i64), P(C.c_double), P(C.c_double), P(C.c_size_t)]),
        "pss_server_destroy": (None, [vp]),
        "pss_sigma_of_power": (C.c_double, [i32, C.c_double]),
        "pss_power_threshold": (C.c_double, [i32, C.c_double]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int, needed: Optional[int] = None):
    if status != PSS_OK:
        raise PssError(status, lib().pss_last_error().decode(), needed)


# ---------------------------------------------------------------------------
# descriptors
# ---------------------------------------------------------------------------

class FilDesc:
    """Keeps a pss_fil_desc and the arrays it points to alive."""

    def __init__(self, nchan, nsamp, tsamp_s, fch0_mhz, foff_mhz, nbits=8, layout=0, chan_mask=None):
        self.mask = None if chan_mask is None else np.ascontiguousarray(chan_mask, dtype=np.uint8)
        self.c = pss_fil_desc(int(nchan), int(nbits), int(nsamp), float(tsamp_s), float(fch0_mhz),
                              float(foff_mhz), int(layout), 0,
                              None if self.mask is None else self.mask.ctypes.data_as(C.POINTER(C.c_uint8)))

    @classmethod
    def of(cls, fil, chan_mask=None, layout=0):
        return cls(fil.nchan, fil.nsamp, fil.tsamp_s, fil.fch0_mhz, fil.foff_mhz, fil.nbits, layout, chan_mask)


def stages_array(stages) -> "C.Array":
    arr = (pss_dd_stage * len(stages))()
    for i, s in enumerate(stages):
        arr[i] = pss_dd_stage(float(s.dm_lo), float(s.dm_step), int(s.n_dm), int(s.ds))
    return arr


def search_cfg(zmax=0, dz=2.0, numharm=8, sigma_thr=6.0, f_lo_hz=1.0, whiten_block=1024, halfwidth_extra=16,
               min_dm_hits=1) -> pss_search_cfg:
    return pss_search_cfg(int(zmax), int(numharm), float(dz), float(sigma_thr), float(f_lo_hz), int(whiten_block),
                          int(halfwidth_extra), int(min_dm_hits), 0)


def cfg_of(c) -> pss_search_cfg:
    return search_cfg(c.zmax, c.dz, c.numharm, c.sigma_thr, c.f_lo_hz, c.whiten_block, c.halfwidth_extra,
                      c.min_dm_hits)


# ---------------------------------------------------------------------------
# objects
# ---------------------------------------------------------------------------

class Context:
    def __init__(self, device: int = 0):
        h = C.c_void_p()
        _check(lib().pss_ctx_create(int(device), C.byref(h)))
        self.h = h
        self.device = device

    def profile(self, enable: bool = True):
        _check(lib().pss_ctx_profile(self.h, int(enable)))

    def profile_read(self):
        """{stage: (ms, launches)} since the last enable/read (synchronises)."""
        ms = np.zeros(len(PROFILE_STAGES), dtype=np.float64)
        n = np.zeros(len(PROFILE_STAGES), dtype=np.int64)
        _check(lib().pss_ctx_profile_read(self.h, ms.ctypes.data, n.ctypes.data))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(PROFILE_STAGES)}

    def close(self):
        if self.h:
            lib().pss_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pss_dd_plan_auto(desc: "FilDesc", dm_lo: float, dm_hi: float, tres_s: float = 0.0, ds_max: int = 1024):
    """Automatic plan rows [(dm_lo, dm_step, n_dm, ds)] for the file shape."""
    cap = 64
    while True:
        out = (pss_dd_stage * cap)()
        n = C.c_int32()
        st = lib().pss_dd_plan_auto(C.byref(desc.c), float(dm_lo), float(dm_hi), float(tres_s), int(ds_max), out,
                                    cap, C.byref(n))
        if st == PSS_ECAP:
            cap = n.value
            continue
        _check(st)
        return [(out[i].dm_lo, out[i].dm_step, out[i].n_dm, out[i].ds) for i in range(n.value)]


class Plan:
    """pss_dd_plan, or pss_dd_plan_subband when subband = (nsub, group)."""

    def __init__(self, desc: FilDesc, stages, subband=None):
        self.desc = desc
        self._st = stages_array(stages)
        h = C.c_void_p()
        if subband is None:
            _check(lib().pss_dd_plan(C.byref(desc.c), self._st, len(stages), C.byref(h)))
        else:
            nsub, group = subband
            _check(lib().pss_dd_plan_subband(C.byref(desc.c), self._st, len(stages), int(nsub), int(group),
                                             C.byref(h)))
        self.h = h
        self.subband = subband
        ndm, dmax = C.c_int64(), C.c_int64()
        _check(lib().pss_plan_info(h, C.byref(ndm), C.byref(dmax), None, None))
        self.ndm, self.max_delay = ndm.value, dmax.value

    def dms(self) -> np.ndarray:
        out = np.empty(self.ndm, dtype=np.float64)
        _check(lib().pss_plan_info(self.h, None, None, out.ctypes.data, None))
        return out

    def delays(self) -> np.ndarray:
        out = np.empty((self.ndm, self.desc.c.nchan), dtype=np.int32)
        _check(lib().pss_plan_info(self.h, None, None, None, out.ctypes.data))
        return out

    def subband_info(self):
        """dict(nsub, group, group_dm [ngroups], chan_delays [ngroups][nchan],
        sub_delays [ndm][nsub]) of a two-stage plan (nsub 0 otherwise)."""
        nsub, group, ng = C.c_int32(), C.c_int32(), C.c_int64()
        _check(lib().pss_plan_subband_info(self.h, C.byref(nsub), C.byref(group), C.byref(ng), None, None, None))
        gdm = np.empty(ng.value, dtype=np.float64)
        e = np.empty((ng.value, self.desc.c.nchan), dtype=np.int32)
        D = np.empty((self.ndm, nsub.value), dtype=np.int32)
        _check(lib().pss_plan_subband_info(self.h, None, None, None, gdm.ctypes.data, e.ctypes.data,
                                           D.ctypes.data))
        return dict(nsub=nsub.value, group=group.value, group_dm=gdm, chan_delays=e, sub_delays=D)

    def trial(self, dm_idx: int):
        s, nv, nfft, ds = C.c_int32(), C.c_int64(), C.c_int64(), C.c_int32()
        _check(lib().pss_plan_trial_info(self.h, int(dm_idx), C.byref(s), C.byref(nv), C.byref(nfft), C.byref(ds)))
        return dict(stage=s.value, nv=nv.value, nfft=nfft.value, ds=ds.value)

    def close(self):
        if self.h:
            lib().pss_plan_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _data_arg(data):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    try:
        import torch
        if isinstance(data, torch.Tensor):
            if not data.is_contiguous():
                raise ValueError("data must be contiguous")
            return C.c_void_p(data.data_ptr()), int(data.is_cuda), data
    except ImportError:
        pass
    arr = np.ascontiguousarray(data)
    return C.c_void_p(arr.ctypes.data), 0, arr


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def _rows(plan: Plan, dm_begin: int, dm_end: int, key: str):
    return [plan.trial(i)[key] for i in range(dm_begin, dm_end)]


# ---------------------------------------------------------------------------
# calls (C names)
# ---------------------------------------------------------------------------

def pss_dedisperse(ctx: Context, plan: Plan, data, dm_begin: int, dm_end: int, out=None, stream=None):
    """int32 device tensor of the packed dedispersed series of [dm_begin, dm_end)."""
    import torch
    total = int(sum(_rows(plan, dm_begin, dm_end, "nv")))
    if out is None:
        out = torch.empty(max(total, 1), dtype=torch.int32, device="cuda:%d" % ctx.device)
    p, dev, keep = _data_arg(data)
    _check(lib().pss_dedisperse(ctx.h, plan.h, C.byref(plan.desc.c), p, dev, dm_begin, dm_end,
                                C.c_void_p(out.data_ptr()), _stream(stream)))
    return out[:total]


def pss_dedisperse_noalloc(plan: Plan, data_dev, dm_begin: int, dm_end: int, out=None, stream=None):
    """pss_dedisperse without device allocation inside the call: data_dev is
    a CUDA tensor, `out` (allocated here if not given, before the call) an
    int32 CUDA tensor of at least sum N_v elements."""
    import torch
    total = int(sum(_rows(plan, dm_begin, dm_end, "nv")))
    if out is None:
        out = torch.empty(max(total, 1), dtype=torch.int32, device=data_dev.device)
    if not (isinstance(data_dev, torch.Tensor) and data_dev.is_cuda):
        raise ValueError("data_dev must be a CUDA tensor")
    _check(lib().pss_dedisperse_noalloc(plan.h, C.byref(plan.desc.c), C.c_void_p(data_dev.data_ptr()), dm_begin,
                                        dm_end, C.c_void_p(out.data_ptr()), _stream(stream)))
    return out[:total]


def pss_single_pulse(ctx: Context, plan: Plan, data, dm_begin: int, dm_end: int, widths=SP_WIDTHS,
                     sigma_thr: float = 6.0, cap: int = 1 << 16, stream=None) -> np.ndarray:
    """Single-pulse events (SP_DTYPE) of trials [dm_begin, dm_end), sorted by
    (dm_idx, t); grows `cap` and calls again when it is too small."""
    p, dev, keep = _data_arg(data)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    while True:
        out = np.zeros(max(cap, 1), dtype=SP_DTYPE)
        n = C.c_int64()
        st = lib().pss_single_pulse(ctx.h, plan.h, C.byref(plan.desc.c), p, dev, dm_begin, dm_end,
                                    w.ctypes.data, len(w), float(sigma_thr), out.ctypes.data, cap, C.byref(n),
                                    _stream(stream))
        if st == PSS_ECAP:
            cap = n.value
            continue
        _check(st)
        return out[: n.value]


def pss_fold(ctx: Context, plan: Plan, data, dm_idx, f_hz, fdot_hz_s=None, nbin: int = 64, nfreq: int = 9,
             step_bins: float = 0.25, stream=None):
    """Fold candidates (arrays of DM index, frequency, drift): (profiles int64
    [n][nbin], counts int64 [n][nbin], results FOLD_RES_DTYPE [n])."""
    dm_idx = np.atleast_1d(np.asarray(dm_idx))
    n = len(dm_idx)
    req = np.zeros(n, dtype=FOLD_REQ_DTYPE)
    req["dm_idx"] = dm_idx
    req["f_hz"] = f_hz
    req["fdot_hz_s"] = 0.0 if fdot_hz_s is None else fdot_hz_s
    prof = np.zeros((n, nbin), dtype=np.int64)
    cnt = np.zeros((n, nbin), dtype=np.int64)
    res = np.zeros(n, dtype=FOLD_RES_DTYPE)
    p, dev, keep = _data_arg(data)
    _check(lib().pss_fold(ctx.h, plan.h, C.byref(plan.desc.c), p, dev, req.ctypes.data, n, nbin, nfreq,
                          float(step_bins), prof.ctypes.data, cnt.ctypes.data, res.ctypes.data, _stream(stream)))
    return prof, cnt, res


def pss_spectrum(ctx: Context, plan: Plan, data, cfg: pss_search_cfg, dm_begin: int, dm_end: int, stream=None):
    """complex64 device tensor: whitened half spectra, rows packed back to back."""
    import torch
    total = int(sum(n // 2 for n in _rows(plan, dm_begin, dm_end, "nfft")))
    out = torch.empty(2 * max(total, 1), dtype=torch.float32, device="cuda:%d" % ctx.device)
    p, dev, keep = _data_arg(data)
    _check(lib().pss_spectrum(ctx.h, plan.h, C.byref(plan.desc.c), p, dev, C.byref(cfg), dm_begin, dm_end,
                              C.c_void_p(out.data_ptr()), _stream(stream)))
    return torch.view_as_complex(out[: 2 * total].view(-1, 2))


def n_z(cfg: pss_search_cfg) -> int:
    return int(round(2 * cfg.zmax / cfg.dz)) + 1 if cfg.zmax else 1


def pss_power_plane(ctx: Context, plan: Plan, data, cfg: pss_search_cfg, dm_begin: int, dm_end: int, stream=None):
    """float32 device tensor: planes [n_z][nfft] of [dm_begin, dm_end) packed back to back."""
    import torch
    nz = n_z(cfg)
    total = int(sum(nz * n for n in _rows(plan, dm_begin, dm_end, "nfft")))
    out = torch.empty(max(total, 1), dtype=torch.float32, device="cuda:%d" % ctx.device)
    p, dev, keep = _data_arg(data)
    _check(lib().pss_power_plane(ctx.h, plan.h, C.byref(plan.desc.c), p, dev, C.byref(cfg), dm_begin, dm_end,
                                 C.c_void_p(out.data_ptr()), _stream(stream)))
    return out[:total]


def pss_search_raw(ctx: Context, plan: Plan, data, cfg: pss_search_cfg, dm_begin: int, dm_end: int,
                   cap: int = 1 << 16, stream=None) -> np.ndarray:
    p, dev, keep = _data_arg(data)
    n = C.c_int64()
    while True:
        out = np.zeros(cap, dtype=RAW_DTYPE)
        st = lib().pss_search_raw(ctx.h, plan.h, C.byref(plan.desc.c), p, dev, C.byref(cfg), dm_begin, dm_end,
                                  out.ctypes.data, cap, C.byref(n), _stream(stream))
        if st == PSS_ECAP:
            cap = n.value
            continue
        _check(st)
        return out[: n.value]


def pss_sift(plan: Plan, cfg: pss_search_cfg, raw: np.ndarray, cap: int = 1 << 14) -> np.ndarray:
    raw = np.ascontiguousarray(raw, dtype=RAW_DTYPE)
    n = C.c_int64()
    while True:
        out = np.zeros(cap, dtype=CAND_DTYPE)
        st = lib().pss_sift(plan.h, C.byref(cfg), raw.ctypes.data, raw.shape[0], out.ctypes.data, cap, C.byref(n))
        if st == PSS_ECAP:
            cap = n.value
            continue
        _check(st)
        return out[: n.value]


def pss_sift_in_batches(plan: Plan, cfg: pss_search_cfg, raw: np.ndarray, dm_bounds, cap: int = 1 << 14) -> np.ndarray:
    raw = np.ascontiguousarray(raw, dtype=RAW_DTYPE)
    bounds = np.ascontiguousarray(dm_bounds, dtype=np.int64)
    n = C.c_int64()
    while True:
        out = np.zeros(cap, dtype=CAND_DTYPE)
        st = lib().pss_sift_in_batches(plan.h, C.byref(cfg), raw.ctypes.data, raw.shape[0], bounds.ctypes.data,
                                       len(bounds) - 1, out.ctypes.data, cap, C.byref(n))
        if st == PSS_ECAP:
            cap = n.value
            continue
        _check(st)
        return out[: n.value]


def pss_search_dm_batch(ctx: Context, plan: Plan, data, cfg: pss_search_cfg, dm_begin: int, dm_end: int,
                        cap: int = 1 << 14, stream=None) -> np.ndarray:
    p, dev, keep = _data_arg(data)
    n = C.c_int64()
    out = np.zeros(cap, dtype=CAND_DTYPE)
    st = lib().pss_search_dm_batch(ctx.h, plan.h, C.byref(plan.desc.c), p, dev, C.byref(cfg), dm_begin, dm_end,
                                   out.ctypes.data, cap, C.byref(n), _stream(stream))
    if st == PSS_ECAP:  # the context kept the list: fetch it without searching again
        out = np.zeros(n.value, dtype=CAND_DTYPE)
        st = lib().pss_ctx_take_cands(ctx.h, out.ctypes.data, n.value, C.byref(n))
    _check(st)
    return out[: n.value]


class pss_multi_file(C.Structure):
    _fields_ = [("plan", C.c_void_p), ("fil", C.POINTER(pss_fil_desc)), ("data", C.c_void_p)]


def _multi_files(files):
    """ctypes array of pss_multi_file for [(Plan, data)], the data all on the
    host or all on the device, and the objects to keep alive meanwhile."""
    arr = (pss_multi_file * len(files))()
    keep, on_dev = [], None
    for k, (plan, data) in enumerate(files):
        p, dev, kp = _data_arg(data)
        if on_dev is None:
            on_dev = dev
        elif on_dev != dev:
            raise ValueError("pss_search_multi: every file on the host, or every file on the device")
        keep.append(kp)
        arr[k].plan = plan.h
        arr[k].fil = C.pointer(plan.desc.c)
        arr[k].data = p.value
    return arr, int(bool(on_dev)), keep


def pss_search_multi(ctx: Context, cfg: pss_search_cfg, files, cap: int = 1 << 14, stream=None):
    """Sifted candidates (CAND_DTYPE) of each of a group of files
    [(Plan, data)] searched together (pss_search_multi): a list, one array
    per file."""
    arr, on_dev, keep = _multi_files(files)
    if on_dev:
        import torch
        torch.cuda.current_stream().synchronize()
    counts = np.zeros(len(files), dtype=np.int64)
    n = C.c_int64()
    out = np.zeros(cap, dtype=CAND_DTYPE)
    st = lib().pss_search_multi(ctx.h, C.byref(cfg), arr, len(files), on_dev, out.ctypes.data, cap,
                                counts.ctypes.data, C.byref(n), _stream(stream))
    if st == PSS_ECAP:  # the context kept the lists: fetch them without searching again
        out = np.zeros(n.value, dtype=CAND_DTYPE)
        st = lib().pss_ctx_take_cands(ctx.h, out.ctypes.data, n.value, C.byref(n))
    _check(st)
    res, off = [], 0
    for c in counts:
        res.append(out[off:off + int(c)])
        off += int(c)
    return res


def pss_search_multi_footprint(cfg: pss_search_cfg, files) -> int:
    arr = (pss_multi_file * len(files))()
    for k, (plan, _) in enumerate(files):
        arr[k].plan = plan.h
        arr[k].fil = C.pointer(plan.desc.c)
    b = C.c_size_t()
    _check(lib().pss_search_multi_footprint(C.byref(cfg), arr, len(files), C.byref(b)))
    return int(b.value)


class Batch:
    """A search prepared for files of one shape and captured into a CUDA
    graph (pss_batch_*); run() searches one file per call."""

    def __init__(self, plan: Plan, cfg: pss_search_cfg, device: int = 0):
        h = C.c_void_p()
        _check(lib().pss_batch_create(int(device), plan.h, C.byref(plan.desc.c), C.byref(cfg), C.byref(h)))
        self.h, self.plan, self.cfg = h, plan, cfg

    @property
    def footprint(self) -> int:
        return int(lib().pss_batch_footprint(self.h))

    @property
    def tuning(self):
        """{fft_split, harm_run, dedisp_kb, whiten_form, fused} chosen by the batch's autotuner."""
        f, h, d, w, u = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        _check(lib().pss_batch_tuning(self.h, C.byref(f), C.byref(h), C.byref(d), C.byref(w), C.byref(u)))
        return {"fft_split": f.value, "harm_run": h.value, "dedisp_kb": d.value, "whiten_form": w.value,
                "fused": u.value}

    def fft_split(self, nfft: int) -> int:
        """The FFT pass split the batch runs for nfft-point series."""
        v = C.c_int32()
        _check(lib().pss_batch_fft_split(self.h, int(nfft), C.byref(v)))
        return v.value

    def run(self, data, cap: int = 1 << 14, timing: bool = False):
        """Sifted candidates of one file (host array or device tensor; a device
        tensor must be complete: the batch copies it on its own stream)."""
        p, dev, keep = _data_arg(data)
        if dev:
            import torch
            torch.cuda.current_stream().synchronize()
        n, ms = C.c_int64(), C.c_double()
        out = np.zeros(cap, dtype=CAND_DTYPE)
        st = lib().pss_batch_run(self.h, p, dev, out.ctypes.data, cap, C.byref(n), C.byref(ms) if timing else None)
        if st == PSS_ECAP:  # the batch kept the list: fetch it without searching again
            out = np.zeros(n.value, dtype=CAND_DTYPE)
            st = lib().pss_batch_take_cands(self.h, out.ctypes.data, n.value, C.byref(n))
        _check(st)
        return (out[: n.value], ms.value) if timing else out[: n.value]

    def close(self):
        if self.h:
            lib().pss_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pss_fft_split_radices(nfft: int, split: int):
    """Pass radices of FFT split `split` for nfft-point series, or None past
    the last split of that size."""
    n = C.c_int32()
    rad = (C.c_int32 * 4)()
    st = lib().pss_fft_split_radices(int(nfft), int(split), C.byref(n), rad)
    if st == PSS_EINVAL:
        return None
    _check(st)
    return [int(rad[i]) for i in range(n.value)]


def pss_fft_splits(nfft: int):
    """Every pass split of the nfft-point FFT: [(split, radices)]."""
    out = []
    for v in range(64):
        r = pss_fft_split_radices(nfft, v)
        if r is None:
            break
        out.append((v, r))
    return out


PEAKS_FIELDS = ["sm_mhz", "add3_per_clk_sm", "lop3_per_clk_sm", "prmt_per_clk_sm", "imad_per_clk_sm",
                "ffma_flops_per_clk_sm", "mix_per_clk_sm", "lds_bytes_per_clk_sm", "int32_adds_per_s", "lop3_per_s",
                "prmt_per_s", "imad_per_s", "fp32_flops_per_s", "mix_per_s", "lds_bytes_per_s"]


class pss_peaks(C.Structure):
    _fields_ = [("sms", C.c_int32), ("reserved", C.c_int32)] + [(n, C.c_double) for n in PEAKS_FIELDS]


def pss_measure_peaks(device: int = 0) -> dict:
    """Measured instruction throughputs of the device (pss_measure_peaks)."""
    p = pss_peaks()
    _check(lib().pss_measure_peaks(int(device), C.byref(p)))
    out = {"sms": int(p.sms)}
    out.update({n: float(getattr(p, n)) for n in PEAKS_FIELDS})
    return out


def pss_ctx_set_wait_limit(ctx: Context, polls: int):
    _check(lib().pss_ctx_set_wait_limit(ctx.h, int(polls)))


def pss_ctx_check(ctx: Context, stream=None):
    _check(lib().pss_ctx_check(ctx.h, _stream(stream)))


def pss_debug_fail_alloc(n: int):
    lib().pss_debug_fail_alloc(int(n))


def pss_ctx_set_fft_split(ctx: Context, nfft: int, split: int):
    _check(lib().pss_ctx_set_fft_split(ctx.h, int(nfft), int(split)))


def pss_batch_create(plan: Plan, cfg: pss_search_cfg, device: int = 0) -> Batch:
    return Batch(plan, cfg, device)


def pss_search_footprint(plan: Plan, cfg: pss_search_cfg) -> int:
    """Device bytes a Batch (or a server slot) for this shape holds."""
    b = C.c_size_t()
    _check(lib().pss_search_footprint(plan.h, C.byref(plan.desc.c), C.byref(cfg), C.byref(b)))
    return int(b.value)


def pss_batch_run(batch: Batch, data, cap: int = 1 << 14) -> np.ndarray:
    return batch.run(data, cap)


class Server:
    """Request loop over files (pss_server_*): submit() queues a file and
    returns a ticket; poll() hands over its candidates once."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 2, device: int = 0, max_group: int = 1):
        """max_group > 1: pss_server_create_grouped (queued files searched in
        groups through pss_search_multi)."""
        h = C.c_void_p()
        _check(lib().pss_server_create_grouped(int(device), C.c_size_t(int(hbm_budget_bytes)), int(max_slots),
                                               int(max_group), C.byref(h)))
        self.h = h

    def submit(self, desc: FilDesc, data, stages, cfg: pss_search_cfg, subband=None) -> int:
        """pss_submit_file, or pss_submit_file_subband when subband = (nsub, group)."""
        arr = np.ascontiguousarray(data, dtype=np.uint8)
        st_arr = stages_array(stages)
        t = C.c_uint64()
        if subband is None:
            _check(lib().pss_submit_file(self.h, C.byref(desc.c), arr.ctypes.data, st_arr, len(stages), C.byref(cfg),
                                         C.byref(t)))
        else:
            _check(lib().pss_submit_file_subband(self.h, C.byref(desc.c), arr.ctypes.data, st_arr, len(stages),
                                                 int(subband[0]), int(subband[1]), C.byref(cfg), C.byref(t)))
        return int(t.value)

    def poll(self, ticket: int, timeout_ms: int = -1):
        """(candidates, latency_s) of a finished file; raises PssError with
        PSS_ENOTREADY / PSS_ETIMEOUT while it is not ready, or the error the
        file met."""
        r = C.c_void_p()
        _check(lib().pss_poll(self.h, C.c_uint64(int(ticket)), int(timeout_ms), C.byref(r)))
        try:
            cp, n, lat = C.c_void_p(), C.c_int64(), C.c_double()
            st = lib().pss_result_cands(r, C.byref(cp), C.byref(n), C.byref(lat))
            _check(st)
            out = np.zeros(n.value, dtype=CAND_DTYPE)
            if n.value:
                C.memmove(out.ctypes.data, cp.value, n.value * CAND_DTYPE.itemsize)
            return out, float(lat.value)
        finally:
            lib().pss_result_free(r)

    def stats(self):
        done, p50, p99, used = C.c_int64(), C.c_double(), C.c_double(), C.c_size_t()
        _check(lib().pss_server_stats(self.h, C.byref(done), C.byref(p50), C.byref(p99), C.byref(used)))
        g, f = C.c_int64(), C.c_int64()
        _check(lib().pss_server_group_stats(self.h, C.byref(g), C.byref(f)))
        return dict(completed=done.value, p50_s=p50.value, p99_s=p99.value, bytes_in_use=int(used.value),
                    groups=g.value, grouped_files=f.value)

    def close(self):
        if self.h:
            lib().pss_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pss_server_create(hbm_budget_bytes: int, max_slots: int = 2, device: int = 0) -> Server:
    return Server(hbm_budget_bytes, max_slots, device)


def pss_refine_prepare(ctx: Context, plan: Plan, data, cfg: pss_search_cfg, stage: int, stream=None):
    p, dev, keep = _data_arg(data)
    _check(lib().pss_refine_prepare(ctx.h, plan.h, C.byref(plan.desc.c), p, dev, C.byref(cfg), int(stage),
                                    _stream(stream)))


def pss_refine_eval(ctx: Context, plan: Plan, points, stream=None):
    """(power [n], grad [n][3]) at refinement points (REFINE_DTYPE array)."""
    pts = np.ascontiguousarray(points, dtype=REFINE_DTYPE)
    n = pts.shape[0]
    power = np.zeros(n, dtype=np.float64)
    grad = np.zeros((n, 3), dtype=np.float64)
    _check(lib().pss_refine_eval(ctx.h, plan.h, pts.ctypes.data, n, power.ctypes.data, grad.ctypes.data,
                                 _stream(stream)))
    return power, grad


def pss_refine_candidates(ctx: Context, plan: Plan, data, cfg: pss_search_cfg, cands: np.ndarray, iters: int = 40,
                          lr: float = 0.05, stream=None) -> np.ndarray:
    out = np.ascontiguousarray(cands, dtype=CAND_DTYPE).copy()
    p, dev, keep = _data_arg(data)
    _check(lib().pss_refine_candidates(ctx.h, plan.h, C.byref(plan.desc.c), p, dev, C.byref(cfg), out.ctypes.data,
                                       out.shape[0], int(iters), float(lr), _stream(stream)))
    return out


def refine_power_function():
    """torch.autograd.Function computing P_h(DM, r, z) on the GPU (after
    pss_refine_prepare) with the library's analytic gradient."""
    import torch

    class RefinePower(torch.autograd.Function):
        @staticmethod
        def forward(fctx, dm, r, z, ctx_, plan, dm_idx, numharm):
            pts = np.zeros(dm.numel(), dtype=REFINE_DTYPE)
            pts["dm_idx"] = np.asarray(dm_idx).reshape(-1)
            pts["numharm"] = np.asarray(numharm).reshape(-1)
            pts["dm"] = dm.detach().cpu().double().numpy().reshape(-1)
            pts["r"] = r.detach().cpu().double().numpy().reshape(-1)
            pts["z"] = z.detach().cpu().double().numpy().reshape(-1)
            power, grad = pss_refine_eval(ctx_, plan, pts)
            g = torch.from_numpy(grad).to(dm.device)
            fctx.save_for_backward(g)
            return torch.from_numpy(power).to(dm.device).reshape(dm.shape)

        @staticmethod
        def backward(fctx, gp):
            (g,) = fctx.saved_tensors
            gp = gp.reshape(-1).double()
            return ((gp * g[:, 0]).reshape(gp.shape), (gp * g[:, 1]).reshape(gp.shape),
                    (gp * g[:, 2]).reshape(gp.shape), None, None, None, None)

    return RefinePower


def pss_response(ctx: Context, q: Sequence[float], z: Sequence[float]) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    out = np.empty(2 * q.shape[0], dtype=np.float64)
    _check(lib().pss_response(ctx.h, q.ctypes.data, z.ctypes.data, q.shape[0], out.ctypes.data))
    return out[0::2] + 1j * out[1::2]


def pss_sigma_of_power(numharm: int, power: float) -> float:
    return lib().pss_sigma_of_power(int(numharm), float(power))


def pss_power_threshold(numharm: int, sigma: float) -> float:
    return lib().pss_power_threshold(int(numharm), float(sigma))


def pss_version() -> str:
    return lib().pss_version().decode()
