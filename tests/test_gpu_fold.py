"""GPU folding (pss_fold) against the oracle (oracle/fold.py) on the same
dedispersed series: identical profiles and counts, the same best trial, and
the reduced chi-square to FP64 rounding."""
import numpy as np
import pytest

from oracle import dedisperse as OD
from oracle import fold as OF
from oracle import plan as OP
from oracle import subband as OSB
from paper_1912_12807_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1912_12807_gb300 import pss
    pss.lib()
    return pss


@pytest.fixture(scope="module")
def ctx(L):
    c = L.Context(0)
    yield c
    c.close()


def _dev(arr):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def _check(L, ctx, fil, stages, dm_idx, f, fdot, nbin, nfreq, step, sub=None):
    plan = L.Plan(L.FilDesc.of(fil), stages, subband=sub)
    op = OP.Plan.for_file(fil, stages, sub)
    x = OD.channel_major(fil.data, fil.nchan, fil.nbits)
    prof, cnt, res = L.pss_fold(ctx, plan, _dev(fil.data), dm_idx, f, fdot, nbin=nbin, nfreq=nfreq, step_bins=step)
    for i, d in enumerate(dm_idx):
        d = int(d)
        ds = int(op.ds_of[d])
        s = (OD.dedisperse(x, op.delays[d], op.max_delay, ds) if sub is None
             else OSB.dedisperse_subband(x, op.sub, d, op.max_delay, ds))
        k, fk, c, P, n = OF.fold_search(s, ds * fil.tsamp_s, op.t_span(d), float(f[i]), float(fdot[i]), nbin, nfreq,
                                        step)
        assert int(res["best"][i]) == k, (i, d)
        assert float(res["f_hz"][i]) == fk
        assert abs(float(res["chi2_red"][i]) - c) <= 1e-12 * max(c, 1.0)
        np.testing.assert_array_equal(prof[i], P)
        np.testing.assert_array_equal(cnt[i], n)
    return prof, cnt, res


def test_fold_small_workload_candidates(L, ctx):
    wl = synth.workload_small()
    T = (1 << 16) * 2e-4
    rng = np.random.default_rng(1)
    dm = np.array([50, 50, 49, 10, 100, 0, 51, 75])
    f = np.array([1 / 0.0333, 2 / 0.0333, 1 / 0.0333, 7.0, 3.3, 1.0, 1 / 0.0333 + 0.3 / T, 123.4])
    fdot = np.array([0.0, 0.0, 0.0, 0.01, -0.02, 0.0, 0.0, 0.0])
    prof, cnt, res = _check(L, ctx, wl.fil, wl.stages, dm, f, fdot, 64, 9, 0.25)
    # the injected 33.3 ms pulsar at DM 50 folds far above the noise trials
    assert res["chi2_red"][0] > 10 * max(res["chi2_red"][3], res["chi2_red"][4])


def test_fold_staged_subband_plan_odd_bins(L, ctx):
    fil = synth.make_1bit(96, 1 << 15, 2.5e-4, 1230.0, 1518.0, [synth.Pulsar(0.02, 100.0, 0.05, 0.1)], seed=4)
    stages = synth.stages_from_table([(0.0, 100.0, 5.0, 1), (100.0, 300.0, 10.0, 2), (300.0, 500.0, 25.0, 4)], True)
    dm = np.array([0, 19, 20, 21, 27, 3])
    f = np.array([50.0, 50.0, 50.0, 100.0, 50.0, 17.0])
    _check(L, ctx, fil, stages, dm, f, np.zeros(6), 37, 5, 0.5, sub=(12, 8))
    _check(L, ctx, fil, stages, dm, f, np.zeros(6), 2, 1, 0.0)


def test_fold_errors(L, ctx):
    wl = synth.workload_small()
    plan = L.Plan(L.FilDesc.of(wl.fil), wl.stages)
    for kw in (dict(nbin=1), dict(nbin=2048), dict(nfreq=0), dict(nfreq=65)):
        with pytest.raises(L.PssError):
            L.pss_fold(ctx, plan, _dev(wl.fil.data), [5], [10.0], **kw)
    with pytest.raises(L.PssError):
        L.pss_fold(ctx, plan, _dev(wl.fil.data), [plan.ndm], [10.0])
