"""Host-side checks of the benchmark: the reference arm's JSON line on the
host cores (the keys every arm prints, the oracle's rate in it, nothing on
the GPU), and the algorithmic work it divides by kernel time."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("small_")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_stage_work_counts_table_terms_and_builds():
    # rows with ds in [8, 256] dedisperse from the boxcar table: one term per channel and
    # output sample (a 32-bit add, two SWAR slots); one table build per distinct ds
    sys.path.insert(0, ROOT)
    import bench
    from paper_1912_12807_gb300 import build, pss, synth
    if not os.path.exists(pss.LIB_PATH):
        build.build()
    wl = synth.workload_fast()
    plan = pss.Plan(pss.FilDesc.of(wl.fil), wl.stages)
    w = bench.stage_work(plan, wl, wl.fil.nbytes())
    C, N = wl.fil.nchan, wl.fil.nsamp
    terms = sum(plan.trial(i)["nv"] for i in range(plan.ndm)) * C
    assert w["dedisperse"] == ("alu", 2.0 * terms, "channel-adds")
    dss = sorted({s.ds for s in wl.stages})
    assert dss == [8, 16, 32, 64, 128]
    build = sum(C * N + 2 * C * ds * (((N + ds - 1) // ds + 7) // 8 * 8) for ds in dss)
    assert w["bxtable"] == ("hbm", float(build), "bytes")
    # a plan of ds 1 rows has no table
    small = synth.workload_small()
    p2 = pss.Plan(pss.FilDesc.of(small.fil), small.stages)
    w2 = bench.stage_work(p2, small, small.fil.nbytes())
    assert w2["bxtable"][1] == 0.0
    assert w2["dedisperse"][1] == float(small.fil.nchan) * sum(p2.trial(i)["nv"] for i in range(p2.ndm))


def test_stage_work_counts_unpack_and_spectrum_bytes():
    # unpack: the file read once plus one byte per channel and sample written (8x the file for
    # 1-bit data); FFT: 16 bytes per complex point and pass; whitening (fused with the zmax 0
    # plane or not): 16 bytes per complex point; zmax 0 plane: 8 M read + 4 nfft written
    sys.path.insert(0, ROOT)
    import math
    import bench
    from paper_1912_12807_gb300 import build, pss, synth
    if not os.path.exists(pss.LIB_PATH):
        build.build()
    small = synth.workload_small()
    plan = pss.Plan(pss.FilDesc.of(small.fil), small.stages)
    w = bench.stage_work(plan, small, small.fil.nbytes())
    C, N = small.fil.nchan, small.fil.nsamp
    assert w["unpack"] == ("hbm", float(C * N + C * N), "bytes")
    Ms = [plan.trial(i)["nfft"] // 2 for i in range(plan.ndm)]
    assert w["fft"] == ("hbm", float(sum(max(1, math.ceil(math.log2(M) / 10)) * 16 * M for M in Ms)), "bytes")
    assert w["whiten"] == ("hbm", float(sum(16 * M for M in Ms)), "bytes")
    assert w["plane"] == ("hbm", float(sum(8 * M + 4 * 2 * M for M in Ms)), "bytes")
    f1 = synth.make_1bit(96, 1 << 15, 2.5e-4, 1230.0, 1518.0, [], seed=1)
    wl1 = synth.Workload("one-bit", f1, [synth.Stage(0.0, 1.0, 8, 1)], small.cfg)
    p1 = pss.Plan(pss.FilDesc.of(f1), wl1.stages)
    w1 = bench.stage_work(p1, wl1, f1.nbytes())
    assert f1.nbytes() * 8 == 96 * (1 << 15)
    assert w1["unpack"] == ("hbm", float(f1.nbytes() + 96 * (1 << 15)), "bytes")
