"""Benchmark: DM-trials searched per second on the drift-scan-shaped file.

Workload (one step): the full periodicity search of one synthetic
256-channel, 2^18-sample (52.4 s at 0.2 ms) 8-bit file over DM 0-500 in
steps of 0.5 (1001 trials), zmax 0, harmonic sums up to 16, 6 sigma:
unpack/transpose, dedispersion, FFT, whitening, power plane, harmonic
sums with thresholding, candidate download and sifting -- one call of
pss_search_dm_batch with the file already resident on the GPU.

`e2e` repeats the step through the same C call with the file in pinned
host memory (upload and candidate download inside the timed region).

Multi-GPU (torchrun): every rank searches its own file (independent
problems, weak scaling, no collective); value = all ranks' DM trials /
the slowest rank's time.

`--impl reference` times the FP64 CPU oracle (the only reference there
is: the paper's pipeline is PRESTO on CPUs, not available here) on the
host cores, on a bounded sample of the same workload's DM trials.
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
WORKLOAD = "driftscan_256ch_2^18_8bit_dm0-500x0.5_1001trials_zmax0_numharm16"
REALTIME_S = 26.0


def _config(extra=None):
    c = {"workload": WORKLOAD, "nchan": 256, "nsamp": 1 << 18, "tsamp_s": 2e-4, "band_mhz": [1050, 1450],
         "dm_trials": 1001, "zmax": 0, "numharm": 16, "sigma_thr": 6.0,
         "l2": "256 MiB buffer written between timed steps (input 64 MiB < L2)"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------- CPU oracle
_W = {}


def _worker_init():
    from paper_1912_12807_gb300 import synth
    from oracle import dedisperse as OD
    from oracle import plan as OP
    from oracle import stats as OST
    wl = synth.workload_driftscan()
    _W["wl"] = wl
    _W["P"] = OP.Plan.for_file(wl.fil, wl.stages)
    _W["x"] = OD.channel_major(wl.fil.data, wl.fil.nchan, 8)
    _W["thr"] = OST.thresholds(wl.cfg.numharm, wl.cfg.sigma_thr)


def _worker_trial(i):
    from oracle import search as OSr
    return len(OSr.search_trial(_W["x"], _W["P"], int(i), _W["wl"].cfg, _W["thr"]))


def _oracle_pool(cores):
    ctx = mp.get_context("spawn")
    return ctx.Pool(cores, initializer=_worker_init)


def oracle_rate(pool, cores, n_trials, ndm=1001, offset=0):
    """Time the oracle over n_trials DM trials spread over the plan."""
    idx = [int((offset + k * ndm / n_trials)) % ndm for k in range(n_trials)]
    t0 = time.perf_counter()
    pool.map(_worker_trial, idx, chunksize=1)
    dt = time.perf_counter() - t0
    return n_trials / dt, dt, idx


def cpu_baseline_block(value, cores, n, dt):
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of the 1001 DM trials (evenly spaced), each searched end to end by the FP64 "
                      "NumPy oracle in a spawn pool of %d processes; %.1f s wall" % (n, cores, dt)}


def run_reference(args, rank):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    pool = _oracle_pool(cores)
    pool.map(_worker_trial, list(range(cores)), chunksize=1)  # warm the workers (imports, file)
    per_step = 4 * cores
    for w in range(args.warmup):
        oracle_rate(pool, cores, cores, offset=w * 7)
    rates, dts = [], []
    for k in range(args.steps):
        r, dt, _ = oracle_rate(pool, cores, per_step, offset=13 + k * 31)
        rates.append(r)
        dts.append(dt)
    pool.close()
    value = per_step * args.steps / sum(dts)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(dts) / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": _config({"step": "%d DM trials per step (bounded sample)" % per_step}),
            "cpu_baseline": cpu_baseline_block(value, cores, per_step * args.steps, sum(dts)),
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


# ---------------------------------------------------------------- GPU arm
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(p)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1912_12807_gb300 import pss, synth

    # CPU baseline first (spawn pool, before any CUDA call), rank 0 at N=1 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        pool = _oracle_pool(cores)
        pool.map(_worker_trial, list(range(cores)), chunksize=1)
        n = 8 * cores
        r, dt, _ = oracle_rate(pool, cores, n, offset=5)
        pool.close()
        cpu = cpu_baseline_block(r, cores, n, dt)

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    wl = synth.workload_driftscan(seed=1002 + rank, n_dm=args.dm_trials)
    fil = wl.fil
    ctx = pss.Context(local_rank)
    plan = pss.Plan(pss.FilDesc.of(fil), wl.stages)
    cfg = pss.cfg_of(wl.cfg)
    ndm = plan.ndm
    data_dev = torch.from_numpy(fil.data).to(dev)
    data_host = torch.from_numpy(fil.data).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(on_device=True):
        src = data_dev if on_device else data_host
        if on_device:
            return pss.pss_search_dm_batch(ctx, plan, src, cfg, 0, ndm, stream=stream.cuda_stream)
        # a numpy view of the pinned tensor: the library uploads it inside the call
        return pss.pss_search_dm_batch(ctx, plan, src.numpy(), cfg, 0, ndm, stream=stream.cuda_stream)

    for _ in range(args.warmup):
        cands = step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # timed region: per-step CUDA events, L2 flushed between steps
    clocks = ClockSampler(local_rank)
    clocks.start()
    ctx.profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        cands = step()
        ev[k][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall0
    prof = ctx.profile_read()
    ctx.profile(False)
    clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms) / len(step_ms)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # e2e through the same call with the file in pinned host memory
    e2e_ms = []
    for k in range(max(1, args.steps)):
        flush.fill_((k + 1) & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = step(on_device=False)
        t1 = time.perf_counter()
        e2e_ms.append(1e3 * (t1 - t0))
    e2e = statistics.mean(e2e_ms)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e = float(t.item())

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    value = world * ndm / (ms / 1e3)
    peaks, peak_kind = measured_peaks()
    d_ms, d_n = prof["dedisperse"]
    launches_per_step = sum(n for _, n in prof.values()) / args.steps
    # dedispersion: C_kept * N_v channel additions per trial (one 8-bit sample
    # added per channel per output sample), all trials of the step in d_n launches
    nv = plan.trial(0)["nv"]
    adds = float(fil.nchan) * nv * ndm
    per_launch_adds = adds * args.steps / max(d_n, 1)
    d_avg_s = (d_ms / max(d_n, 1)) / 1e3
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    # ALU ceiling of the SWAR scheme: 152 SMs x 64 integer-ALU lanes per clock
    # x 2 sixteen-bit additions per 32-bit add, at the maximum SM clock
    alu_peak = 152 * 64 * 2 * sm_mhz * 1e6
    achieved = per_launch_adds / d_avg_s if d_avg_s > 0 else 0.0
    roof = {"kernel": "k_dedisp", "bound": "alu", "achieved": achieved / 1e12, "peak": alu_peak / 1e12,
            "unit": "T channel-adds/s", "frac": achieved / alu_peak, "traffic": None,
            "peak_source": "derived: 152 SMs x 64 INT lanes x 2 (16-bit SWAR) x %.0f MHz (%s clock)"
                           % (sm_mhz, peak_kind)}
    bi = fil.nbytes()
    bo = int(len(cands)) * pss.CAND_DTYPE.itemsize
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i32+f32", "data": "synthetic",
            "config": _config({"dm_trials": ndm}), "files_per_s": world * 1e3 / ms, "s_per_file": ms / 1e3,
            "realtime_budget_s": REALTIME_S, "realtime_factor": REALTIME_S / (ms / 1e3),
            "roofline": roof,
            "e2e": {"value": world * ndm / (e2e / 1e3), "unit": UNIT, "h2d_bytes_per_step": bi,
                    "d2h_bytes_per_step": bo, "ms_per_step": e2e},
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "stages_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "stage_launches_per_step": {k: v[1] / args.steps for k, v in prof.items()},
            "clocks": clocks.summary(), "wall_s_timed": t_wall, "candidates": int(len(cands)),
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--dm-trials", type=int, default=1001,
                    help="DM trials of the plan (0.5 step from DM 0); smaller values make profiling cases")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
