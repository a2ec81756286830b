"""GPU parity on the FAST-shaped file (200 channels over 290-340 MHz, 2^18 x
0.2 ms, 8-bit) with the paper's Table 3 plan (979 trials, six rows, ds 8 to
128, nfft 2^15 down to 2^11), in the launch configuration the benchmark
times: every trial of the plan in one call; sampled trials (each row's first
and last, and the trials nearest the injected pulsars) checked against the
oracle: the int32 series bit for bit, the raw candidates set for set."""
import numpy as np
import pytest

from oracle import dedisperse as OD
from oracle import plan as OP
from paper_1912_12807_gb300 import synth

from _parity import compare_candidates, oracle_plane

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


@pytest.fixture(scope="module")
def fast():
    wl = synth.workload_fast()
    op = OP.Plan.for_file(wl.fil, wl.stages)
    x = OD.channel_major(wl.fil.data, wl.fil.nchan, 8)
    edges = np.cumsum([0] + [s.n_dm for s in wl.stages])
    sample = set()
    for k in range(len(wl.stages)):
        sample |= {int(edges[k]), int(edges[k + 1]) - 1}
    for p in wl.fil.pulsars:
        sample.add(int(np.argmin(np.abs(op.dms - p.dm))))
    return wl, op, x, sorted(sample)


def _dev(arr):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def test_fast_table3_dedisperse_sampled(L, ctx, fast):
    wl, op, x, sample = fast
    plan = L.Plan(L.FilDesc.of(wl.fil), wl.stages)
    assert plan.ndm == 979 and plan.max_delay == op.max_delay
    out = L.pss_dedisperse(ctx, plan, _dev(wl.fil.data), 0, plan.ndm).cpu().numpy()
    off = 0
    for i in range(plan.ndm):
        nv, _ = op.nv_nfft(i)
        if i in sample:
            ref = OD.dedisperse(x, op.delays[i], op.max_delay, int(op.ds_of[i]))
            np.testing.assert_array_equal(out[off:off + nv], ref, err_msg="DM index %d" % i)
        off += nv
    assert off == out.shape[0]


def test_fast_table3_search_sampled(L, ctx, fast):
    wl, op, x, sample = fast
    plan = L.Plan(L.FilDesc.of(wl.fil), wl.stages)
    cfg = L.cfg_of(wl.cfg)
    raw = L.pss_search_raw(ctx, plan, _dev(wl.fil.data), cfg, 0, plan.ndm)
    tot = 0
    for i in sample:
        _, _, pl = oracle_plane(x, op, i, wl.cfg)
        g, r, e = compare_candidates(raw, pl, i, wl.cfg.numharm, 0, op.t_span(i), wl.cfg.f_lo_hz,
                                     wl.cfg.sigma_thr)
        tot += r
    assert tot > 50
    # the sifted list of the whole plan is the sift of the raw list
    cands = L.pss_search_dm_batch(ctx, plan, _dev(wl.fil.data), cfg, 0, plan.ndm)
    assert cands.tobytes() == L.pss_sift(plan, cfg, raw).tobytes()
