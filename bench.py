"""Benchmark: DM-trials searched per second.

Default workload (one step): the full periodicity search of one synthetic
256-channel, 2^18-sample (52.4 s at 0.2 ms) 8-bit drift-scan-shaped file
over DM 0-500 in steps of 0.5 (1001 trials), zmax 0, harmonic sums up to 16,
6 sigma: unpack/transpose, dedispersion, FFT, whitening, power plane,
harmonic sums with thresholding, candidate download and sifting -- one call
of pss_search_dm_batch with the file already resident on the GPU.

Other workloads (--workload): accel (same file shape, DM 0-300 step 1,
zmax 200, dz 2, numharm 8), pmps (96-channel 1-bit 2^23-sample file, staged
plan of 1081 trials, zmax 0, numharm 16), pmps50 (the same with zmax 50),
small (64 channels, 2^16 samples, 101 trials).

`e2e` repeats the step through the same C call with the file in pinned
host memory (upload and candidate download inside the timed region).
`batched` runs the same file through a prepared, graph-captured search
(pss_batch); `serve` streams files of the same shape through the request
loop (pss_server): saturated throughput, and p50/p99 latency at paced
arrivals.

Multi-GPU (torchrun): every rank searches its own file (independent
problems, weak scaling, no collective); value = all ranks' DM trials /
the slowest rank's time.

`--impl reference` times the FP64 CPU oracle (the only reference there is:
the paper's pipeline is PRESTO on CPUs, not available here) on the host
cores, on a bounded sample of the same workload's DM trials.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DM-trials searched/s and files/s vs 26 s realtime; batched vs plain; p99 lat"
UNIT = "DM-trials/s"
REALTIME_S = 26.0
OLA_L = 2048  # overlap-save segment of the zmax > 0 plane
BX_MIN = int(os.environ.get("PSS_DEDISP_BX_MIN") or "8")  # rows with ds >= this use the boxcar table (0: none)

WORKLOADS = {
    "driftscan": "driftscan_256ch_2^18_8bit_dm0-500x0.5_1001trials_zmax0_numharm16",
    "accel": "accel_256ch_2^18_8bit_dm0-300x1_301trials_zmax200_dz2_numharm8",
    "pmps": "pmps_96ch_1bit_2^23_staged1081trials_zmax0_numharm16",
    "pmps50": "pmps_96ch_1bit_2^23_staged1081trials_zmax50_numharm16",
    "small": "small_64ch_2^16_8bit_dm0-100x1_101trials_zmax0_numharm8",
    "fast": "fast_200ch_290-340MHz_2^18_8bit_table3_979trials_ds8-128_zmax0_numharm16",
}
# The paper's own number for the FAST-shaped file: 979 trials in 166 s on 24
# CPU cores (whole pipeline; Sect. 3.3); context only, another machine.
PAPER_RATE = {"fast": 979.0 / 166.0}


def make_workload(name: str, n_dm=None, seed_offset: int = 0):
    from paper_1912_12807_gb300 import synth
    if name == "driftscan":
        return synth.workload_driftscan(seed=1002 + seed_offset, n_dm=n_dm or 1001)
    if name == "accel":
        return synth.workload_accel(seed=1003 + seed_offset, n_dm=n_dm or 301)
    if name == "pmps":
        return synth.workload_pmps(seed=1004 + seed_offset, zmax=0)
    if name == "pmps50":
        return synth.workload_pmps(seed=1004 + seed_offset, zmax=50)
    if name == "small":
        return synth.workload_small(seed=1001 + seed_offset)
    if name == "fast":
        return synth.workload_fast(seed=1006 + seed_offset)
    raise ValueError(name)


def _config(wl, name, extra=None):
    f = wl.fil
    c = {"workload": WORKLOADS[name], "nchan": f.nchan, "nsamp": f.nsamp, "nbits": f.nbits,
         "tsamp_s": f.tsamp_s, "dm_trials": int(sum(s.n_dm for s in wl.stages)),
         "stages": [[s.dm_lo, s.dm_step, s.n_dm, s.ds] for s in wl.stages],
         "zmax": wl.cfg.zmax, "dz": wl.cfg.dz, "numharm": wl.cfg.numharm, "sigma_thr": wl.cfg.sigma_thr,
         "l2": "256 MiB buffer written between timed steps"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------- CPU oracle
_W = {}


def _worker_init(name):
    from oracle import dedisperse as OD
    from oracle import plan as OP
    from oracle import stats as OST
    wl = make_workload(name)
    _W["wl"] = wl
    _W["P"] = OP.Plan.for_file(wl.fil, wl.stages)
    _W["x"] = OD.channel_major(wl.fil.data, wl.fil.nchan, wl.fil.nbits)
    _W["thr"] = OST.thresholds(wl.cfg.numharm, wl.cfg.sigma_thr)


def _worker_trial(i):
    from oracle import search as OSr
    method = "fftconv" if _W["wl"].cfg.zmax > 0 else "direct"
    return len(OSr.search_trial(_W["x"], _W["P"], int(i), _W["wl"].cfg, _W["thr"], plane_method=method))


def _oracle_pool(cores, name):
    ctx = mp.get_context("spawn")
    return ctx.Pool(cores, initializer=_worker_init, initargs=(name,))


def oracle_rate(pool, n_trials, ndm, offset=0):
    """Time the oracle over n_trials DM trials spread over the plan."""
    idx = [int((offset + k * ndm / n_trials)) % ndm for k in range(n_trials)]
    t0 = time.perf_counter()
    pool.map(_worker_trial, idx, chunksize=1)
    dt = time.perf_counter() - t0
    return n_trials / dt, dt


def cpu_baseline_block(value, cores, n, ndm, dt):
    which = ("%d of the %d DM trials (evenly spaced)" % (n, ndm) if n <= ndm else
             "%d trial searches cycling evenly over the %d DM trials" % (n, ndm))
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%s, each searched end to end by the FP64 NumPy oracle in a spawn pool of %d "
                      "processes; %.1f s wall" % (which, cores, dt)}


def _per_step_trials(name, cores):
    # keep a sample near 10-30 s of CPU work
    per_core = {"driftscan": 8, "small": 40, "accel": 1, "pmps": 1, "pmps50": 1, "fast": 40}[name]
    return max(2, per_core * cores)


def run_reference(args, rank):
    if rank != 0:
        return
    name = args.workload
    wl = make_workload(name)
    ndm = int(sum(s.n_dm for s in wl.stages))
    cores = os.cpu_count() or 1
    pool = _oracle_pool(cores, name)
    pool.map(_worker_trial, list(range(min(cores, ndm))), chunksize=1)  # warm the workers
    per_step = max(1, _per_step_trials(name, cores) // 2)
    for w in range(args.warmup):
        oracle_rate(pool, max(1, cores // 2), ndm, offset=w * 7)
    dts = []
    for k in range(args.steps):
        _, dt = oracle_rate(pool, per_step, ndm, offset=13 + k * 31)
        dts.append(dt)
    pool.close()
    value = per_step * args.steps / sum(dts)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(dts) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": _config(wl, name, {"step": "%d DM trials per step (bounded sample)" % per_step}),
            "cpu_baseline": cpu_baseline_block(value, cores, per_step * args.steps, ndm, sum(dts)),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, n in enumerate(names):
                if s[5 + k].lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------- rooflines
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def max_over_ranks(x, world, device=None):
    """The largest value of x over all ranks (the slowest rank's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, trials_per_rank, ms):
    """Whole-job DM-trials/s: every rank searches its own file (weak scaling)."""
    return world * trials_per_rank / (ms / 1e3)


def recorded_traffic(workload, stage):
    """DRAM bytes per launch of a stage's kernel from the committed ncu capture
    (profiles/dram_traffic.json), or None when there is none or the kernel
    source has changed since it was taken."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        rec = json.load(open(p))[workload][stage]
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
    except (OSError, KeyError, ValueError):
        return None
    if hashlib.sha1(src).hexdigest() != rec["source_sha1"]:
        return None
    return float(rec["dram_read_bytes"]) + float(rec["dram_write_bytes"])


def bx_row(plan, wl, stage):
    """Whether the library dedisperses a plan stage from the boxcar table when
    the whole plan is searched in one call: ds in [BX_MIN, 256], an exact
    plan, at most 65535 kept channels, and at least 16 trials in the row."""
    st = wl.stages[stage]
    return (BX_MIN > 0 and BX_MIN <= st.ds <= 256 and st.n_dm >= 16 and wl.fil.nchan <= 65535
            and not getattr(plan, "subband", None))


def stage_work(plan, wl, fil_nbytes):
    """Algorithmic work of one step per profiled stage: (bound, amount, unit).

    dedisperse: kept channels x output samples x ds additions (each output
    sample sums one 8-bit sample per channel per native sample), two 16-bit
    SWAR additions per 32-bit add; rows that dedisperse from the boxcar table
    add one 16-bit table term per channel and output sample with one 32-bit
    add, counted as the two SWAR slots it takes; bxtable: the table builds;
    unpack: file read + channel-major write; fft: every pass reads and writes
    8 bytes per complex point; whiten: spectrum read + write (where the
    whitening and the zmax 0 plane run as one kernel, the stage reads the
    spectrum and writes the plane: the same bytes, and the plane stage has
    no launches); plane: for
    zmax 0 the spectrum read + plane write, for zmax > 0 the flops of the
    overlap-save correlation (5 L log2 L per L-point FFT, 6 per complex
    product) or, where the direct form runs, the 8 flops of every complex tap;
    harmsum: one read of the plane."""
    ndm = plan.ndm
    cfg = wl.cfg
    nz = int(round(2 * cfg.zmax / cfg.dz)) + 1 if cfg.zmax else 1
    adds = 0.0
    fft_b = whiten_b = plane_b = harm_b = 0.0
    plane_flops = 0.0
    for i in range(ndm):
        t = plan.trial(i)
        nv, nfft, ds = t["nv"], t["nfft"], t["ds"]
        M = nfft // 2
        if bx_row(plan, wl, t["stage"]):
            adds += 2.0 * wl.fil.nchan * nv  # one 32-bit add per table term: two SWAR add slots
        else:
            adds += float(wl.fil.nchan) * nv * ds
        passes = max(1, int(math.ceil(math.log2(M) / 10)))
        fft_b += passes * 2 * 8.0 * M
        whiten_b += 2 * 8.0 * M
        harm_b += 4.0 * nz * nfft
        if cfg.zmax == 0:
            plane_b += 8.0 * M + 4.0 * nfft
        else:
            mmax = (cfg.zmax + 1) // 2 + cfg.halfwidth_extra
            if 4 * mmax <= OLA_L and M >= OLA_L:
                # overlap-save: per segment of OLA_L bins, one forward FFT, then per
                # row two pointwise products and two FFTs (5 L log2 L flops each)
                V = OLA_L - 2 * mmax + 1
                fft = 5.0 * OLA_L * math.log2(OLA_L)
                plane_flops += math.ceil(M / V) * (fft + nz * 2 * (6.0 * OLA_L + fft))
            else:
                for j in range(nz):
                    z = -cfg.zmax + j * cfg.dz
                    m = int(math.ceil(abs(z) / 2)) + cfg.halfwidth_extra
                    plane_flops += 2 * (2 * m) * 8.0 * M
    # boxcar-table builds (rows with ds in [BX_MIN, 256]): one per distinct ds, reading the
    # channel-major bytes and writing the uint16 table of C x ds x ceil(N/ds) (rows of 8)
    C, N = wl.fil.nchan, wl.fil.nsamp
    bx_b = 0.0
    for ds in sorted({s.ds for k, s in enumerate(wl.stages) if bx_row(plan, wl, k)}):
        mstride = ((N + ds - 1) // ds + 7) // 8 * 8
        bx_b += float(C) * N + 2.0 * C * ds * mstride
    # unpack: the file read once, one byte per channel and sample written (8x the file for 1-bit data)
    return {"unpack": ("hbm", float(fil_nbytes) + float(wl.fil.nchan) * wl.fil.nsamp, "bytes"),
            "dedisperse": ("alu", adds, "channel-adds"),
            "bxtable": ("hbm", bx_b, "bytes"),
            "fft": ("hbm", fft_b, "bytes"),
            "whiten": ("hbm", whiten_b, "bytes"),
            "plane": ("hbm", plane_b, "bytes") if cfg.zmax == 0 else ("alu", plane_flops, "flops"),
            "harmsum": ("hbm", harm_b, "bytes")}


# Instructions per channel-addition at the floor of the SWAR dedispersion loop:
# per 32-bit word of 4 samples one 128-bit shared-memory load serves 4 words
# (0.25), two extractions (mask and byte permute) and one three-input add that
# folds two channels' halves (1.0): 3.25 instructions per 4 channel-additions.
DEDISP_INSTR_PER_ADD = 3.25 / 4.0


def alu_denominators(probe):
    """Integer and FP32 roofline denominators from the device probes
    (pss_measure_peaks): the dedispersion ceiling is the smaller of the
    shared-memory operand bandwidth (every channel-addition reads its 8-bit
    sample from shared memory once: 1 byte) and the issue rate with the
    integer and FMA pipes busy over DEDISP_INSTR_PER_ADD instructions."""
    smem = probe["lds_bytes_per_s"]
    issue = probe["mix_per_s"] / DEDISP_INSTR_PER_ADD
    return {"channel_adds_per_s": min(smem, issue), "smem_bound_adds_per_s": smem,
            "issue_bound_adds_per_s": issue, "int32_adds_per_s": probe["int32_adds_per_s"],
            "fp32_flops_per_s": probe["fp32_flops_per_s"]}


def roofline_of(stage, bound, amount, unit, ms, launches, peaks, peak_kind, alu):
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    per_launch = amount / max(launches, 1)
    t = (ms / max(launches, 1)) / 1e3
    ach = per_launch / t if t > 0 else 0.0
    if bound == "hbm":
        peak = hbm * 1e9
        return {"kernel": stage, "bound": "hbm", "achieved": ach / 1e9, "peak": hbm, "unit": "GB/s",
                "frac": ach / peak, "traffic": None, "peak_source": "hbm_gbs (%s)" % peak_kind}
    if unit == "channel-adds":
        peak = alu["channel_adds_per_s"]
        return {"kernel": stage, "bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12,
                "unit": "T channel-adds/s", "frac": ach / peak, "traffic": None,
                "frac_of_int32_add_peak": ach / (2.0 * alu["int32_adds_per_s"]),
                "peak_source": "measured (pss_measure_peaks): min(shared-memory load bytes/s at 1 byte per "
                               "channel-add, lop3/imad issue rate / %.4f instructions per channel-add)"
                               % DEDISP_INSTR_PER_ADD}
    peak = alu["fp32_flops_per_s"]
    return {"kernel": stage, "bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": ach / peak, "traffic": None, "peak_source": "measured (pss_measure_peaks): FP32 FMA rate"}


# ---------------------------------------------------------------- GPU arm
def measure_search(pss, wl, name, steps, warmup, local_rank, flush, stream, peaks, peak_kind, alu, world=1,
                   traffic=True):
    """One workload through pss_search_dm_batch with the file resident on
    the device: `steps` steps timed by CUDA events on the launching stream
    (L2 flushed between them), per-stage device time from the library's
    profiler in up to 3 further steps (its events stay out of the timed
    ones), rooflines against the measured peaks, then the same call with
    the file in pinned host memory (upload and candidate download timed).
    Returns (result dict, context, plan, cfg, device data, candidates); the
    caller closes the context."""
    import torch
    dev = torch.device("cuda", local_rank)
    fil = wl.fil
    ctx = pss.Context(local_rank)
    plan = pss.Plan(pss.FilDesc.of(fil), wl.stages)
    cfg = pss.cfg_of(wl.cfg)
    ndm = plan.ndm
    data_dev = torch.from_numpy(fil.data).to(dev)
    data_host = torch.from_numpy(fil.data).pin_memory()

    def step(on_device=True):
        if on_device:
            return pss.pss_search_dm_batch(ctx, plan, data_dev, cfg, 0, ndm, stream=stream.cuda_stream)
        # a numpy view of the pinned tensor: the library uploads it inside the call
        return pss.pss_search_dm_batch(ctx, plan, data_host.numpy(), cfg, 0, ndm, stream=stream.cuda_stream)

    cands = None
    for _ in range(warmup):
        cands = step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier()
    t_wall0 = time.perf_counter()
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        cands = step()
        ev[k][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)
    # the stage breakdown from further steps with the library's per-stage CUDA events on
    # (kept out of the timed steps: the events are instrumentation, not the search)
    psteps = max(1, min(steps, 3))
    ctx.profile(True)
    for k in range(psteps):
        flush.fill_(k & 0xFF)
        step()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)

    e2e_ms = []
    for k in range(max(1, steps)):
        flush.fill_((k + 1) & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(on_device=False)
        t1 = time.perf_counter()
        e2e_ms.append(1e3 * (t1 - t0))
    e2e = max_over_ranks(statistics.mean(e2e_ms), world, dev)

    work = stage_work(plan, wl, fil.nbytes())
    rooflines = {}
    for st, (ms_st, n_st) in prof.items():
        if n_st == 0:
            continue
        bound, amount, unit = work[st]
        rooflines[st] = roofline_of(st, bound, amount * psteps, unit, ms_st, n_st, peaks, peak_kind, alu)
        if traffic:
            rooflines[st]["traffic"] = recorded_traffic(name, st)
    if "whiten" in rooflines and cfg.zmax == 0 and prof.get("plane", (0.0, 0))[1] == 0:
        rooflines["whiten"]["note"] = ("whitening and the zmax 0 plane in one kernel (k_whiten_z0, k_z0_seams): "
                                       "spectrum read, plane written")
    if "dedisperse" in rooflines:
        # the same launches against HBM: every trial's FP32 series written once, the
        # channel-major file read once per launch
        ms_dd, n_dd = prof["dedisperse"]
        nv_sum = sum(plan.trial(i)["nv"] for i in range(ndm))
        dd_bytes = 4.0 * nv_sum * psteps + float(fil.nchan) * fil.nsamp * n_dd
        rooflines["dedisperse"]["hbm_frac"] = (dd_bytes / (ms_dd / 1e3)) / (float(peaks.get("hbm_gbs", 6800.0)) * 1e9)
        bx_rows = sorted({wl.stages[k].ds for k in range(len(wl.stages)) if bx_row(plan, wl, k)})
        if bx_rows:
            rooflines["dedisperse"]["note"] = (
                "rows with ds %s dedisperse from a per-channel boxcar table built once per ds (stage bxtable): "
                "one table term per output and channel, a 32-bit add counted as two 16-bit SWAR slots" % bx_rows)
    dominant = max(prof, key=lambda k: prof[k][0])
    launches_per_step = sum(n for _, n in prof.values()) / psteps
    bi = fil.nbytes()
    bo = int(len(cands)) * pss.CAND_DTYPE.itemsize
    res = {"metric": METRIC, "value": job_value(world, ndm, ms), "unit": UNIT, "steps": steps, "warmup": warmup,
           "ms_per_step": ms, "config": _config(wl, name, {"dm_trials": ndm}), "files_per_s": world * 1e3 / ms,
           "s_per_file": ms / 1e3, "realtime_budget_s": REALTIME_S, "realtime_factor": REALTIME_S / (ms / 1e3),
           "roofline": rooflines[dominant],
           "e2e": {"value": job_value(world, ndm, e2e), "unit": UNIT, "h2d_bytes_per_step": bi,
                   "d2h_bytes_per_step": bo, "ms_per_step": e2e},
           "gpu_launches": int(round(launches_per_step * steps)),
           "stages_ms_per_step": {k: v[0] / psteps for k, v in prof.items()},
           "stage_launches_per_step": {k: v[1] / psteps for k, v in prof.items()},
           "stage_rooflines": {k: {kk: v[kk] for kk in ("bound", "frac", "achieved", "unit", "hbm_frac", "note")
                                   if kk in v} for k, v in rooflines.items()},
           "clocks": clocks.summary(), "wall_s_timed": t_wall, "candidates": int(len(cands))}
    return res, ctx, plan, cfg, data_dev, cands


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1912_12807_gb300 import pss

    name = args.workload
    # CPU baseline first (spawn pool, before any CUDA call), rank 0 at N=1 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        wl0 = make_workload(name)
        ndm0 = int(sum(s.n_dm for s in wl0.stages))
        cores = os.cpu_count() or 1
        pool = _oracle_pool(cores, name)
        pool.map(_worker_trial, list(range(min(cores, ndm0))), chunksize=1)
        n = _per_step_trials(name, cores)
        r, dt = oracle_rate(pool, n, ndm0, offset=5)
        pool.close()
        cpu = cpu_baseline_block(r, cores, n, ndm0, dt)

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    peaks, peak_kind = measured_peaks()
    probe = pss.pss_measure_peaks(local_rank)
    alu = alu_denominators(probe)
    wl = make_workload(name, n_dm=args.dm_trials, seed_offset=rank)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    head, ctx, plan, cfg, data_dev, cands = measure_search(
        pss, wl, name, args.steps, args.warmup, local_rank, flush, stream, peaks, peak_kind, alu, world,
        traffic=args.dm_trials is None)
    ndm = plan.ndm

    refine = None
    if wl.cfg.zmax > 0 and rank == 0 and len(cands) and args.refine_top > 0:
        refine = run_refine(pss, ctx, plan, data_dev, cfg, cands, args.refine_top)

    subband = None
    if args.subband != "none" and rank == 0:
        nsub, group = (int(v) for v in args.subband.split(","))
        subband = run_subband(pss, ctx, wl, data_dev, cfg, ndm, max(3, args.steps), flush, stream, cands,
                              nsub, group)

    folded = None
    if args.fold_top > 0 and rank == 0 and len(cands):
        folded = run_fold(pss, ctx, plan, data_dev, cands, args.fold_top, max(3, args.steps))

    single = None
    if args.single_pulse and rank == 0:
        single = run_single_pulse(pss, ctx, plan, data_dev, ndm, max(3, args.steps), flush)

    batched = served = None
    if not args.no_serve:
        batched = run_batched(pss, plan, cfg, data_dev, ndm, max(3, args.steps), flush)
        if rank == 0:
            served = run_served(pss, name, wl, args, local_rank)
    ctx.close()
    del data_dev

    # the other workloads of the benchmark, each a sub-object with its own timing (1 GPU only)
    extras = {}
    if rank == 0 and world == 1 and args.extras:
        for ex in args.extras.split(","):
            t0 = time.perf_counter()
            if ex == "stream":
                extras["stream"] = run_stream(args, local_rank, n_files=args.extra_stream_files)
            else:
                extras[ex] = run_extra(pss, ex, args, local_rank, flush, stream, peaks, peak_kind, alu)
            extras[ex]["bench_wall_s"] = time.perf_counter() - t0

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": head["value"] / PAPER_RATE[name] if name in PAPER_RATE and args.dm_trials is None else None,
            "dtype": "i32+f32", "data": "synthetic"}
    for k in ("config", "files_per_s", "s_per_file", "realtime_budget_s", "realtime_factor", "roofline", "e2e",
              "gpu_launches", "stages_ms_per_step", "stage_launches_per_step", "stage_rooflines", "clocks",
              "wall_s_timed", "candidates"):
        line[k] = head[k]
    line.update({"batched": batched, "serve": served, "refine": refine, "subband": subband, "single_pulse": single,
                 "fold": folded, "alu_peaks": {"probe": probe, "denominators": alu}, "cpu_baseline": cpu})
    line.update(extras)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_extra(pss, ex, args, local_rank, flush, stream, peaks, peak_kind, alu):
    """A sub-object of the default line: the acceleration file with the
    refinement of its top 4096 candidates and its prepared batch (accel), the
    PMPS-shaped file at zmax 0 and 50 (pmps), or the FAST-shaped file with the
    printed Table 3 plan (fast)."""
    import torch
    steps = max(2, args.extra_steps)
    if ex == "accel":
        wl = make_workload("accel")
        res, ctx, plan, cfg, data_dev, cands = measure_search(pss, wl, "accel", steps, 3, local_rank, flush, stream,
                                                              peaks, peak_kind, alu)
        if len(cands) and args.refine_top > 0:
            res["refine"] = run_refine(pss, ctx, plan, data_dev, cfg, cands, args.refine_top)
        ctx.close()
        res["batched"] = run_batched(pss, plan, cfg, data_dev, plan.ndm, steps, flush)
        return res
    if ex == "pmps":
        wl = make_workload("pmps")
        out = {}
        for z, key in ((0, "zmax0"), (50, "zmax50")):
            wl.cfg.zmax = z
            nm = "pmps" if z == 0 else "pmps50"
            res, ctx, plan, cfg, data_dev, cands = measure_search(pss, wl, nm, steps, 3 if z == 0 else 2, local_rank,
                                                                  flush, stream, peaks, peak_kind, alu)
            ctx.close()
            out[key] = res
            del data_dev
            torch.cuda.empty_cache()
        return out
    if ex == "fast":
        wl = make_workload("fast")
        res, ctx, plan, cfg, data_dev, cands = measure_search(pss, wl, "fast", max(steps, 5), 3, local_rank, flush,
                                                              stream, peaks, peak_kind, alu)
        ctx.close()
        res["vs_paper_cpu_rate"] = res["value"] / PAPER_RATE["fast"]
        return res
    raise ValueError(ex)


def run_refine(pss, ctx, plan, data_dev, cfg, cands, top, iters=40):
    """Continuous (DM, r, z) refinement of the `top` highest-sigma candidates
    by gradient ascent (pss_refine_candidates): wall time of the call (which
    prepares the per-channel spectra of each candidate stage, then runs the
    ascent), and how much the refined power exceeds the search's."""
    import numpy as np
    import torch
    sel = cands[np.argsort(-cands["sigma"], kind="stable")[:top]]
    pss.pss_refine_candidates(ctx, plan, data_dev, cfg, sel[: min(8, len(sel))], iters=2)  # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = pss.pss_refine_candidates(ctx, plan, data_dev, cfg, sel, iters=iters)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    gain = out["power"] / np.maximum(sel["power"], 1e-30)
    return {"candidates": int(len(sel)), "iters": iters, "s": dt, "cands_per_s": len(sel) / dt,
            "power_gain_median": float(np.median(gain)), "power_gain_min": float(gain.min()),
            "stages_prepared": int(len(np.unique([plan.trial(int(i))["stage"] for i in sel["dm_idx"]])))}


def run_subband(pss, ctx, wl, data_dev, cfg, ndm, steps, flush, stream, exact, nsub, group):
    """The same search on a two-stage (subband) plan of the same DM grid
    (pss_dd_plan_subband): device time per file (CUDA events, L2 flushed
    between steps), the dedispersion stage time, and how many of the exact
    search's sifted candidates it finds again (same frequency within 1.5
    bins of the span, DM within 2 steps)."""
    import numpy as np
    import torch
    plan = pss.Plan(pss.FilDesc.of(wl.fil), wl.stages, subband=(nsub, group))
    for _ in range(3):
        cands = pss.pss_search_dm_batch(ctx, plan, data_dev, cfg, 0, ndm, stream=stream.cuda_stream)
    torch.cuda.synchronize()
    ctx.profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_((k + 3) & 0xFF)
        ev[k][0].record(stream)
        cands = pss.pss_search_dm_batch(ctx, plan, data_dev, cfg, 0, ndm, stream=stream.cuda_stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    dms = plan.dms()
    step = float(np.min(np.diff(dms))) if len(dms) > 1 else 1.0
    T = wl.fil.nsamp * wl.fil.tsamp_s
    found = 0
    for c in exact:
        m = (np.abs(cands["f_hz"] - c["f_hz"]) <= 1.5 / T) & (np.abs(cands["dm"] - c["dm"]) <= 2 * step + 1e-9)
        found += bool(m.any())
    max_delay = plan.max_delay
    plan.close()
    return {"nsub": nsub, "group": group, "value": ndm / (ms / 1e3), "unit": UNIT, "ms_per_file": ms,
            "stages_ms_per_file": {k: v[0] / steps for k, v in prof.items()},
            "stage_launches_per_file": {k: v[1] / steps for k, v in prof.items()},
            "candidates": int(len(cands)), "exact_candidates_found": found, "exact_candidates": int(len(exact)),
            "max_delay": max_delay}


def run_fold(pss, ctx, plan, data_dev, cands, top, steps, nbin=64, nfreq=9, step_bins=0.25):
    """Folding (pss_fold) of the `top` highest-sigma sifted candidates on a grid
    of nfreq trial frequencies each: wall time per call, which includes the
    exact dedispersion of the candidates' trials."""
    import numpy as np
    import torch
    sel = cands[np.argsort(-cands["sigma"], kind="stable")[:top]]
    fdot = np.array([float(c["z"]) / plan.trial(int(c["dm_idx"]))["nfft"] ** 2 /
                     (plan.trial(int(c["dm_idx"]))["ds"] * plan.desc.c.tsamp_s) ** 2 for c in sel])
    args = (ctx, plan, data_dev, sel["dm_idx"], sel["f_hz"], fdot)
    pss.pss_fold(*args, nbin=nbin, nfreq=nfreq, step_bins=step_bins)
    dts = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, res = pss.pss_fold(*args, nbin=nbin, nfreq=nfreq, step_bins=step_bins)
        dts.append(time.perf_counter() - t0)
    w = statistics.mean(dts)
    return {"candidates": int(len(sel)), "trial_freqs": nfreq, "nbin": nbin, "wall_ms": 1e3 * w,
            "cands_per_s": len(sel) / w, "distinct_trials": int(len(np.unique(sel["dm_idx"]))),
            "chi2_red_median": float(np.median(res["chi2_red"]))}


def run_single_pulse(pss, ctx, plan, data_dev, ndm, steps, flush):
    """Single-pulse search (pss_single_pulse: exact int32 dedispersion of every
    trial, boxcar detection on the device, S/N and pruning on the host) over
    the whole file: wall time per file with the event download."""
    import torch
    pss.pss_single_pulse(ctx, plan, data_dev, 0, ndm)
    dts, n = [], 0
    for k in range(steps):
        flush.fill_((k + 5) & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev = pss.pss_single_pulse(ctx, plan, data_dev, 0, ndm)
        dts.append(time.perf_counter() - t0)
        n = len(ev)
    w = statistics.mean(dts)
    return {"value": ndm / w, "unit": UNIT, "wall_ms_per_file": 1e3 * w, "events": n,
            "widths": list(pss.SP_WIDTHS), "sigma_thr": 6.0}


def run_batched(pss, plan, cfg, data_dev, ndm, steps, flush):
    """The same file through a prepared, graph-captured pss_batch: one graph
    launch per file (device time from the batch's own events; wall time
    includes the candidate download and the host sift)."""
    import torch
    b = pss.Batch(plan, cfg)
    for _ in range(3):
        b.run(data_dev)
    gpu, wall = [], []
    for k in range(steps):
        flush.fill_((k + 7) & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, g = b.run(data_dev, timing=True)
        wall.append(time.perf_counter() - t0)
        gpu.append(g)
    fp = b.footprint
    tuning = b.tuning
    b.close()
    g, w = statistics.mean(gpu), statistics.mean(wall)
    return {"value": ndm / (g / 1e3), "unit": UNIT, "gpu_ms_per_file": g, "wall_ms_per_file": 1e3 * w,
            "wall_dm_trials_per_s": ndm / w, "launches_per_file": "1 graph", "device_bytes": fp,
            "tuning": tuning}


def run_served(pss, name, wl, args, device):
    """A stream of files of the workload's shape (distinct contents) through the
    request loop (pss_server): (a) all submitted at once, for throughput
    with the host sift of one file overlapping the kernels of the next;
    (b) paced arrivals, for submit-to-result latency percentiles."""
    import numpy as np
    n_distinct, n_files = 4, max(16, 4 * args.steps)
    # distinct contents of one shape: the file rotated in time
    datas = [np.ascontiguousarray(np.roll(wl.fil.data, 40503 * i, axis=0)) for i in range(n_distinct)]
    desc = pss.FilDesc.of(wl.fil)
    cfg = pss.cfg_of(wl.cfg)
    ndm = int(sum(s.n_dm for s in wl.stages))
    slots = args.serve_slots
    srv = pss.Server(int(args.serve_budget_gib * (1 << 30)), max_slots=slots, device=device)
    # warm-up at the same queue depth: batches prepared, pinned staging pool grown
    for t in [srv.submit(desc, datas[i % n_distinct], wl.stages, cfg) for i in range(n_files)]:
        srv.poll(t)
    t0 = time.perf_counter()
    ts = [srv.submit(desc, datas[i % n_distinct], wl.stages, cfg) for i in range(n_files)]
    t_sub = time.perf_counter() - t0
    for t in ts:
        srv.poll(t)
    dt = time.perf_counter() - t0
    # paced (same server, batches prepared): arrivals every `gap` seconds (about half the measured capacity)
    gap = 2.0 * dt / n_files
    lat = []
    tick = time.perf_counter()
    pending = []
    for i in range(n_files):
        while time.perf_counter() < tick + i * gap:
            time.sleep(gap / 20)
        pending.append(srv.submit(desc, datas[i % n_distinct], wl.stages, cfg))
    for t in pending:
        lat.append(srv.poll(t)[1])
    srv.close()
    lat.sort()
    pct = lambda q: lat[max(0, math.ceil(q / 100.0 * len(lat)) - 1)]
    return {"slots": slots, "files": n_files, "distinct_files": n_distinct,
            "saturated": {"value": n_files * ndm / dt, "unit": UNIT, "files_per_s": n_files / dt,
                          "realtime_factor": REALTIME_S * n_files / dt, "submit_ms_per_file": 1e3 * t_sub / n_files},
            "paced": {"arrival_gap_ms": 1e3 * gap, "p50_ms": 1e3 * pct(50), "p99_ms": 1e3 * pct(99),
                      "max_ms": 1e3 * lat[-1]},
            "budget_gib": args.serve_budget_gib}


def run_stream(args, local_rank, n_files=None):
    """Mixed-shape drift-scan stream (128-1024 channels, 2^17-2^19 samples,
    0-3 pulsars, DM 0-500 step 1, zmax 100, numharm 8; Poisson arrivals with
    a 26 s mean replayed faster by --stream-speedup): the plain per-file loop
    (pss_search_dm_batch on host data, one file after another), then the
    request loop (pss_server) saturated (all files queued at once) and paced
    at the replayed arrival times, with submit-to-result latencies.  Returns
    the measurement as a dict (the contract keys included)."""
    import torch

    from paper_1912_12807_gb300 import pss, synth
    n_files = n_files or args.stream_files
    torch.cuda.set_device(local_rank)
    t0 = time.perf_counter()
    files = list(synth.stream_files(n_files, speedup=args.stream_speedup))
    t_gen = time.perf_counter() - t0
    ndm = int(sum(st.n_dm for st in files[0][1].stages))
    shapes = sorted({(w.fil.nchan, w.fil.nsamp) for _, w in files})
    descs = [pss.FilDesc.of(w.fil) for _, w in files]
    cfg = pss.cfg_of(files[0][1].cfg)
    stages = files[0][1].stages
    # plain loop: one context, one file after another (each shape warmed once first)
    ctx = pss.Context(local_rank)
    plans = {}
    for (_, w), d in zip(files, descs):
        key = (w.fil.nchan, w.fil.nsamp)
        if key not in plans:
            plans[key] = pss.Plan(d, stages)
            pss.pss_search_dm_batch(ctx, plans[key], w.fil.data, cfg, 0, ndm)
    clocks = ClockSampler(local_rank)
    clocks.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_plain = 0
    for (_, w) in files:
        c = pss.pss_search_dm_batch(ctx, plans[(w.fil.nchan, w.fil.nsamp)], w.fil.data, cfg, 0, ndm)
        n_plain += len(c)
    t_plain = time.perf_counter() - t0
    ctx.close()
    budget = int(args.serve_budget_gib * (1 << 30))
    # served, saturated: every file queued at once (after one warm pass that prepares the batches)
    srv = pss.Server(budget, max_slots=args.serve_slots, device=local_rank)
    for t in [srv.submit(d, w.fil.data, stages, cfg) for (_, w), d in zip(files, descs)]:
        srv.poll(t)
    t0 = time.perf_counter()
    ts = [srv.submit(d, w.fil.data, stages, cfg) for (_, w), d in zip(files, descs)]
    n_served = sum(len(srv.poll(t)[0]) for t in ts)
    t_sat = time.perf_counter() - t0
    # served, paced at the replayed arrival times
    tick = time.perf_counter()
    pending = []
    for (ta, w), d in zip(files, descs):
        while time.perf_counter() < tick + ta:
            time.sleep(0.001)
        pending.append(srv.submit(d, w.fil.data, stages, cfg))
    lat = sorted(srv.poll(t)[1] for t in pending)
    t_paced = time.perf_counter() - tick
    srv.close()
    # grouped: queued files searched together (pss_search_multi: one launch per stage over a group)
    grouped = None
    if args.stream_group > 1:
        srv = pss.Server(budget, max_slots=args.serve_slots, device=local_rank, max_group=args.stream_group)
        for t in [srv.submit(d, w.fil.data, stages, cfg) for (_, w), d in zip(files, descs)]:
            srv.poll(t)
        t0 = time.perf_counter()
        ts = [srv.submit(d, w.fil.data, stages, cfg) for (_, w), d in zip(files, descs)]
        n_grouped = sum(len(srv.poll(t)[0]) for t in ts)
        t_gsat = time.perf_counter() - t0
        st_sat = srv.stats()
        tick = time.perf_counter()
        pending = []
        for (ta, w), d in zip(files, descs):
            while time.perf_counter() < tick + ta:
                time.sleep(0.001)
            pending.append(srv.submit(d, w.fil.data, stages, cfg))
        glat = sorted(srv.poll(t)[1] for t in pending)
        t_gpaced = time.perf_counter() - tick
        st_all = srv.stats()
        srv.close()
        gp = lambda q: glat[max(0, math.ceil(q / 100.0 * len(glat)) - 1)]
        grouped = {"max_group": args.stream_group, "slots": args.serve_slots,
                   "saturated": {"value": len(files) * ndm / t_gsat, "unit": UNIT, "files_per_s": len(files) / t_gsat,
                                 "s_per_file": t_gsat / len(files)},
                   "paced": {"p50_ms": 1e3 * gp(50), "p99_ms": 1e3 * gp(99), "max_ms": 1e3 * glat[-1],
                             "wall_s": t_gpaced},
                   "groups": st_all["groups"], "grouped_files": st_all["grouped_files"],
                   "groups_saturated_pass": st_sat["groups"], "candidates": n_grouped}
    clocks.stop()
    pct = lambda q: lat[max(0, math.ceil(q / 100.0 * len(lat)) - 1)]
    n = len(files)
    value = n * ndm / t_sat
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": n, "warmup": n,
            "ms_per_step": 1e3 * t_sat / n, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "i32+f32", "data": "synthetic",
            "config": {"workload": "stream_%dfiles_128-1024ch_2^17-2^19_dm0-500x1_zmax100_numharm8" % n,
                       "files": n, "shapes": [list(x) for x in shapes], "dm_trials_per_file": ndm,
                       "zmax": cfg.zmax, "numharm": cfg.numharm, "arrival_mean_s": 26.0,
                       "replay_speedup": args.stream_speedup, "slots": args.serve_slots,
                       "budget_gib": args.serve_budget_gib, "input": "host memory (copied at submit)"},
            "files_per_s": n / t_sat, "realtime_factor": REALTIME_S * n / t_sat,
            "plain": {"value": n * ndm / t_plain, "unit": UNIT, "files_per_s": n / t_plain,
                      "s_per_file": t_plain / n},
            "served_saturated": {"value": value, "unit": UNIT, "files_per_s": n / t_sat, "s_per_file": t_sat / n},
            "served_paced": {"p50_ms": 1e3 * pct(50), "p99_ms": 1e3 * pct(99), "max_ms": 1e3 * lat[-1],
                             "wall_s": t_paced, "realtime_budget_s": REALTIME_S},
            "candidates": {"plain": n_plain, "served": n_served},
            "grouped": grouped,
            "clocks": clocks.summary(), "generation_s": t_gen}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="driftscan", choices=sorted(WORKLOADS) + ["stream"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="skip the batched and served measurements")
    ap.add_argument("--serve-slots", type=int, default=2)
    ap.add_argument("--serve-budget-gib", type=float, default=64.0)
    ap.add_argument("--stream-files", type=int, default=64)
    ap.add_argument("--refine-top", type=int, default=4096, help="candidates refined after a zmax > 0 search")
    ap.add_argument("--stream-speedup", type=float, default=50.0)
    ap.add_argument("--stream-group", type=int, default=16,
                    help="files per group of the grouped server in the stream measurement (1: not measured)")
    ap.add_argument("--fold-top", type=int, default=64, help="sifted candidates folded after the search (0: none)")
    ap.add_argument("--single-pulse", type=int, default=None,
                    help="1: also time the single-pulse search of every trial (default: 1 for the drift-scan workload)")
    ap.add_argument("--subband", default=None,
                    help="'nsub,group' of a two-stage plan searched beside the exact one, or 'none' "
                         "(default: 16,16 for the drift-scan workload, none otherwise)")
    ap.add_argument("--extras", default=None,
                    help="comma list of other workloads measured as sub-objects of the default line at N=1 "
                         "(accel, pmps, stream, fast; default: all four for the drift-scan workload, none otherwise; "
                         "'' for none)")
    ap.add_argument("--extra-steps", type=int, default=3, help="timed steps of each extra workload")
    ap.add_argument("--extra-stream-files", type=int, default=16, help="files of the extra stream measurement")
    ap.add_argument("--dm-trials", type=int, default=None,
                    help="DM trials of a single-stage plan (driftscan/accel); smaller values make profiling cases")
    args = ap.parse_args()
    if args.subband is None:
        args.subband = "16,16" if args.workload == "driftscan" else "none"
    if args.single_pulse is None:
        args.single_pulse = 1 if args.workload == "driftscan" else 0
    if args.extras is None:
        args.extras = "accel,pmps,stream,fast" if args.workload == "driftscan" and args.dm_trials is None else ""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.workload == "stream":
        if rank == 0:
            print(json.dumps(run_stream(args, local_rank)), flush=True)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
