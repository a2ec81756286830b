"""Alternative kernel forms chosen per process (environment) give the same
bytes: the double- and single-buffered FFT passes (PSS_FFT_DB, with the
shared-memory sub-stage passes, PSS_FFT_RR=0) and zmax 0 plane kernels
(PSS_PLANE_Z0_DB), the whitening fused with the zmax 0 plane against
the two kernels (PSS_WHITEN_Z0), the unpack kernels for files with
every channel kept against the tiled one (PSS_PREP_FAST), and the
register-radix FFT passes with staged double-buffered tiles against the
unstaged ones (PSS_FFT_STAGE).  The register-radix FFT passes (PSS_FFT_RR=1, the
default) round differently: both FFT forms are compared with the oracle."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1912_12807_gb300 import pss, synth
wl = synth.workload_small(nsamp={nsamp})
ctx = pss.Context(0)
plan = pss.Plan(pss.FilDesc.of(wl.fil), wl.stages)
cfg = pss.cfg_of(wl.cfg)
d = torch.from_numpy(wl.fil.data).cuda()
spec = pss.pss_spectrum(ctx, plan, d, cfg, 0, 40).cpu().numpy()
plane = pss.pss_power_plane(ctx, plan, d, cfg, 0, 40).cpu().numpy()
np.save({out!r}, np.concatenate([spec.ravel().view(np.float32), plane.ravel().view(np.float32)]))
"""


def _run(tmp_path, env_extra, nsamp, tag):
    out = str(tmp_path / ("spec_%s.npy" % tag))
    env = dict(os.environ)
    env.update(env_extra)
    subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT, nsamp=nsamp, out=out)], env=env, check=True,
                   timeout=600)
    return np.load(out)


@pytest.mark.parametrize("nsamp", [1 << 16, (1 << 16) + 12345])
def test_fft_and_plane_forms_are_bit_identical(tmp_path, nsamp):
    a = _run(tmp_path, {"PSS_FFT_RR": "0", "PSS_FFT_DB": "0", "PSS_PLANE_Z0_DB": "0"}, nsamp, "single")
    b = _run(tmp_path, {"PSS_FFT_RR": "0", "PSS_FFT_DB": "1", "PSS_FFT_TPC": "3", "PSS_PLANE_Z0_TPC": "3"}, nsamp,
             "double")
    assert a.shape == b.shape and a.tobytes() == b.tobytes()


@pytest.mark.parametrize("nsamp", [1 << 16, (1 << 15) + 777])
def test_fft_register_and_shared_forms_match_oracle(tmp_path, nsamp):
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from _parity import check_powers, oracle_plane
    from oracle import dedisperse as OD
    from oracle import plan as OP
    from paper_1912_12807_gb300 import synth
    wl = synth.workload_small(nsamp=nsamp)
    op = OP.Plan.for_file(wl.fil, wl.stages)
    x = OD.channel_major(wl.fil.data, wl.fil.nchan, 8)
    M = op.nv_nfft(0)[1] // 2
    refs = [np.abs(oracle_plane(x, op, i, wl.cfg)[1]) ** 2 for i in range(40)]
    for tag, env in (("rr", {"PSS_FFT_RR": "1"}), ("smem", {"PSS_FFT_RR": "0"})):
        got = _run(tmp_path, env, nsamp, tag)
        spec = got[: 2 * 40 * M].view(np.complex64)
        for i in range(40):
            check_powers(np.abs(spec[i * M:(i + 1) * M]) ** 2, refs[i], "%s form, trial %d" % (tag, i))


CHILD_Z0 = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1912_12807_gb300 import pss, synth
out = []
for nsamp, W in {cases!r}:
    wl = synth.workload_small(nsamp=nsamp)
    ctx = pss.Context(0)
    plan = pss.Plan(pss.FilDesc.of(wl.fil), wl.stages)
    cfg = pss.search_cfg(zmax=0, numharm=8, whiten_block=W)
    d = torch.from_numpy(wl.fil.data).cuda()
    out.append(pss.pss_power_plane(ctx, plan, d, cfg, 0, 40).cpu().numpy().ravel().view(np.uint8))
    out.append(pss.pss_search_dm_batch(ctx, plan, d, cfg, 0, plan.ndm).view(np.uint8))
    ctx.close()
np.save({out!r}, np.concatenate(out))
"""


def test_whitening_fused_with_zmax0_plane_is_bit_identical(tmp_path):
    # whitening blocks of 1024, 512 and 256 bins (4 blocks per CTA range: several interior range
    # boundaries), a ragged series, and a spectrum of two blocks (a CTA with idle warp pairs)
    cases = [(1 << 16, 1024), ((1 << 16) + 12345, 512), (1 << 15, 256), (3000, 1024)]
    outs = []
    for tag, v in (("fused", "1"), ("separate", "0")):
        out = str(tmp_path / ("z0_%s.npy" % tag))
        env = dict(os.environ)
        env["PSS_WHITEN_Z0"] = v
        subprocess.run([sys.executable, "-c", CHILD_Z0.format(root=ROOT, cases=cases, out=out)], env=env,
                       check=True, timeout=600)
        outs.append(np.load(out))
    assert outs[0].size > 0 and outs[0].tobytes() == outs[1].tobytes()


CHILD_PREP = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1912_12807_gb300 import pss, synth
out = []
files = [synth.make_8bit(64, 40000 + 7, 2e-4, 1200.0, 1500.0, [synth.Pulsar(0.02, 30.0, 0.05, 0.5)], seed=5),
         synth.make_8bit(260, 30000, 2e-4, 1200.0, 1500.0, [], seed=6),
         synth.make_1bit(96, 50000 + 33, 2.5e-4, 1230.0, 1518.0, [synth.Pulsar(0.02, 100.0, 0.05, 0.1)], seed=7)]
for fil in files:
    ctx = pss.Context(0)
    plan = pss.Plan(pss.FilDesc.of(fil), [synth.Stage(0.0, 2.0, 40, 1)])
    d = torch.from_numpy(fil.data).cuda()
    out.append(pss.pss_dedisperse(ctx, plan, d, 0, plan.ndm).cpu().numpy().ravel().view(np.uint8))
    ctx.close()
np.save({out!r}, np.concatenate(out))
"""


def test_unpack_forms_are_identical(tmp_path):
    # 8-bit files of 64 and 260 channels (ragged series) and a 1-bit file of 96 channels: the
    # register-transpose and ballot unpack kernels against the tiled one, through dedispersion
    outs = []
    for tag, v in (("fast", "1"), ("tiled", "0")):
        out = str(tmp_path / ("prep_%s.npy" % tag))
        env = dict(os.environ)
        env["PSS_PREP_FAST"] = v
        subprocess.run([sys.executable, "-c", CHILD_PREP.format(root=ROOT, out=out)], env=env, check=True,
                       timeout=600)
        outs.append(np.load(out))
    assert outs[0].size > 0 and outs[0].tobytes() == outs[1].tobytes()


CHILD_STAGE = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1912_12807_gb300 import pss, synth
out = []
for nsamp in {cases!r}:
    wl = synth.workload_small(nsamp=nsamp)
    ctx = pss.Context(0)
    plan = pss.Plan(pss.FilDesc.of(wl.fil), [synth.Stage(0.0, 1.0, 24, 1)])
    cfg = pss.search_cfg(zmax=0, numharm=8, whiten_block=256)
    d = torch.from_numpy(wl.fil.data).cuda()
    out.append(pss.pss_spectrum(ctx, plan, d, cfg, 0, plan.ndm).cpu().numpy().ravel().view(np.uint8))
    ctx.close()
np.save({out!r}, np.concatenate(out))
"""


def test_fft_staged_tiles_are_bit_identical(tmp_path):
    # complex transforms of 2^11 (radix 64 x 32), 2^15 (256 x 128), 2^16 with a ragged series
    # (256 x 256) and 2^21 (128 x 128 x 128) points: the staged first and later passes against
    # k_fft_pass_rr
    cases = [2500, 1 << 16, (1 << 16) + 12345, (1 << 22) + 77]
    outs = []
    for tag, v in (("staged", "1"), ("direct", "0")):
        out = str(tmp_path / ("stage_%s.npy" % tag))
        env = dict(os.environ)
        env["PSS_FFT_STAGE"] = v
        env["PSS_FFT_STAGE_LATER"] = v  # every pass staged (the default stages the first only)
        env["PSS_FFT_RR"] = "1"
        subprocess.run([sys.executable, "-c", CHILD_STAGE.format(root=ROOT, cases=cases, out=out)], env=env,
                       check=True, timeout=900)
        outs.append(np.load(out))
    assert outs[0].size > 0 and outs[0].tobytes() == outs[1].tobytes()


CHILD_DD = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1912_12807_gb300 import pss, synth
sys.path.insert(0, {tests!r})
from test_gpu_forms import dd_case
fil, stages = dd_case()
ctx = pss.Context(0)
plan = pss.Plan(pss.FilDesc.of(fil), stages)
d = torch.from_numpy(fil.data).cuda()
a = pss.pss_dedisperse(ctx, plan, d, 0, plan.ndm).cpu().numpy()
b = pss.pss_dedisperse(ctx, plan, d, 40, 95).cpu().numpy()
np.save({out!r}, np.concatenate([a.ravel(), b.ravel()]))
"""


def dd_case():
    """48 channels x 40000 samples; rows of ds 1 to 512, most with 16 or more
    trials (a call takes the boxcar table for a row of ds in [PSS_DEDISP_BX_MIN,
    256] when it has at least 16 of its trials)."""
    from paper_1912_12807_gb300 import synth
    fil = synth.make_8bit(48, 40000, 2e-4, 1200.0, 1500.0, [synth.Pulsar(0.01, 30.0, 0.05, 0.5)], seed=11)
    stages = [synth.Stage(0.0, 2.0, 5, 1), synth.Stage(10.0, 2.0, 16, 2), synth.Stage(42.0, 3.0, 16, 4),
              synth.Stage(90.0, 4.0, 16, 8), synth.Stage(154.0, 5.0, 17, 16), synth.Stage(239.0, 20.0, 16, 128),
              synth.Stage(559.0, 30.0, 16, 256), synth.Stage(1039.0, 40.0, 2, 512)]
    return fil, stages


def test_dedisp_boxcar_table_and_direct_forms_are_identical(tmp_path):
    # rows with ds in [PSS_DEDISP_BX_MIN, 256] dedisperse from the boxcar table; 0 turns it off
    from oracle import dedisperse as OD
    from oracle import plan as OP
    outs = []
    for tag, v in (("direct", "0"), ("table2", "2"), ("default", None)):
        out = str(tmp_path / ("dd_%s.npy" % tag))
        env = dict(os.environ)
        env.pop("PSS_DEDISP_BX_MIN", None)
        if v is not None:
            env["PSS_DEDISP_BX_MIN"] = v
        child = CHILD_DD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), out=out)
        subprocess.run([sys.executable, "-c", child], env=env, check=True, timeout=600)
        outs.append(np.load(out))
    assert outs[0].tobytes() == outs[1].tobytes() == outs[2].tobytes()
    # and the first and last trial of every row equal the oracle's series
    fil, stages = dd_case()
    op = OP.Plan.for_file(fil, stages)
    x = OD.channel_major(fil.data, fil.nchan, 8)
    off, first = 0, 0
    for st in stages:
        for i in range(first, first + st.n_dm):
            nv, _ = op.nv_nfft(i)
            if i in (first, first + st.n_dm - 1):
                ref = OD.dedisperse(x, op.delays[i], op.max_delay, st.ds)
                np.testing.assert_array_equal(outs[1][off:off + nv], ref, err_msg="DM index %d" % i)
            off += nv
        first += st.n_dm


CHILD_SEARCH = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_1912_12807_gb300 import pss, synth
sys.path.insert(0, {tests!r})
from test_gpu_forms import search_cases
res = []
for fil, stages, mask in search_cases():
    ctx = pss.Context(0)
    plan = pss.Plan(pss.FilDesc.of(fil, chan_mask=mask), stages)
    cfg = pss.search_cfg(zmax=0, numharm=8)
    d = torch.from_numpy(fil.data).cuda()
    spec = pss.pss_spectrum(ctx, plan, d, cfg, 0, plan.ndm).cpu().numpy()
    raw = pss.pss_search_raw(ctx, plan, d, cfg, 0, plan.ndm)
    res.append(spec.view(np.float32).ravel())
    res.append(np.frombuffer(raw.tobytes(), dtype=np.float32))
    ctx.close()
np.save({out!r}, np.concatenate(res))
"""


def search_cases():
    """A masked 8-bit file and a 1-bit file, each with rows of ds 8 to 128 of
    16 or more trials (the boxcar-table path of the search: float series with
    per-trial sums)."""
    from paper_1912_12807_gb300 import synth
    f8 = synth.make_8bit(64, 1 << 18, 2e-4, 1200.0, 1500.0, [synth.Pulsar(0.05, 40.0, 0.05, 0.6)], seed=21)
    mask = np.ones(64, dtype=np.uint8)
    mask[[1, 2, 30, 63]] = 0
    st8 = [synth.Stage(0.0, 4.0, 16, 8), synth.Stage(64.0, 6.0, 18, 32), synth.Stage(172.0, 10.0, 16, 128)]
    f1 = synth.make_1bit(96, 1 << 17, 2.5e-4, 1230.0, 1518.0, [synth.Pulsar(0.1, 80.0, 0.05, 0.1)], seed=22)
    st1 = [synth.Stage(0.0, 5.0, 16, 8), synth.Stage(80.0, 10.0, 20, 16), synth.Stage(280.0, 20.0, 16, 64)]
    return [(f8, st8, mask), (f1, st1, None)]


def test_dedisp_boxcar_table_search_path_is_identical(tmp_path):
    # the search's float series and per-trial sums through the table equal the direct kernel's:
    # identical spectra and raw candidates, masked 8-bit and 1-bit files
    outs = []
    for tag, v in (("direct", "0"), ("table", "2")):
        out = str(tmp_path / ("srch_%s.npy" % tag))
        env = dict(os.environ)
        env["PSS_DEDISP_BX_MIN"] = v
        child = CHILD_SEARCH.format(root=ROOT, tests=os.path.join(ROOT, "tests"), out=out)
        subprocess.run([sys.executable, "-c", child], env=env, check=True, timeout=600)
        outs.append(np.load(out))
    assert outs[0].size > 0 and outs[0].tobytes() == outs[1].tobytes()
