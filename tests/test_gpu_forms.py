"""Alternative kernel forms chosen per process (environment) give the same
bytes: the double- and single-buffered FFT passes (PSS_FFT_DB) and zmax 0
plane kernels (PSS_PLANE_Z0_DB)."""
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
    a = _run(tmp_path, {"PSS_FFT_DB": "0", "PSS_PLANE_Z0_DB": "0"}, nsamp, "single")
    b = _run(tmp_path, {"PSS_FFT_DB": "1", "PSS_FFT_TPC": "3", "PSS_PLANE_Z0_TPC": "3"}, nsamp, "double")
    assert a.shape == b.shape and a.tobytes() == b.tobytes()
