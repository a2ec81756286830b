"""GPU parity of the two-stage (subband) dedispersion, through the C ABI,
against the oracle's two-stage scheme (oracle/subband.py): bit-exact int32
series; and the search on a two-stage plan against the oracle search on the
same plan."""
import numpy as np
import pytest

from oracle import dedisperse as OD
from oracle import plan as OP
from oracle import subband as OSB
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
def small():
    return synth.workload_small()


def _dev(arr):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


def _check(L, ctx, fil, stages, sub, mask=None, layout=0, rng_=None, trials=None):
    desc = L.FilDesc.of(fil, chan_mask=mask, layout=layout)
    plan = L.Plan(desc, stages, subband=sub)
    op = OP.Plan.for_file(fil, stages, sub)
    assert plan.max_delay == op.max_delay
    x = OD.channel_major(fil.data, fil.nchan, fil.nbits)
    data = fil.data if layout == 0 else x
    b, e = rng_ if rng_ else (0, plan.ndm)
    out = L.pss_dedisperse(ctx, plan, _dev(data), b, e).cpu().numpy()
    off = 0
    for i in range(b, e):
        nv, _ = op.nv_nfft(i)
        if trials is None or i in trials:
            ref = OSB.dedisperse_subband(x, op.sub, i, op.max_delay, int(op.ds_of[i]), mask)
            np.testing.assert_array_equal(out[off:off + nv], ref, err_msg="DM index %d" % i)
        off += nv
    assert off == out.shape[0]
    return plan, out


@pytest.mark.parametrize("sub", [(8, 8), (16, 5), (4, 40), (1, 16)])
def test_subband_small_bit_exact(L, ctx, small, sub):
    _check(L, ctx, small.fil, small.stages, sub)


def test_subband_mask_subrange_channel_major(L, ctx, small):
    mask = np.ones(64, dtype=np.uint8)
    mask[[0, 7, 8, 40, 63]] = 0
    mask[16:24] = 0  # one whole subband of 8 removed
    _check(L, ctx, small.fil, small.stages, (8, 8), mask=mask, rng_=(30, 70))  # starts mid-group
    _check(L, ctx, small.fil, small.stages, (8, 6), layout=1, rng_=(3, 29))


def test_one_channel_subbands_equal_exact_gpu(L, ctx, small):
    fil = small.fil
    exact = L.pss_dedisperse(ctx, L.Plan(L.FilDesc.of(fil), small.stages), _dev(fil.data), 0, 101).cpu().numpy()
    plan, out = _check(L, ctx, fil, small.stages, (64, 16), trials={0, 50, 100})
    np.testing.assert_array_equal(out, exact)


@pytest.mark.parametrize("nchan,nsamp,ds,sub", [(48, 20000 + 37, 1, (6, 5)), (300, 9000 + 5, 1, (12, 16)),
                                                (64, 40000 + 11, 4, (16, 3)), (32, 33333, 1024, (4, 16)),
                                                (300, 9000 + 5, 2, (1, 1))])
def test_subband_ragged_wide_downsampled(L, ctx, nchan, nsamp, ds, sub):
    fil = synth.make_8bit(nchan, nsamp, 2e-4, 1200.0, 1500.0, [synth.Pulsar(0.05, 30.0, 0.05, 0.8)], seed=nchan)
    stages = [synth.Stage(0.0, 3.0, 13, 1), synth.Stage(39.0, 7.0, 9, ds)]
    _check(L, ctx, fil, stages, sub)


def test_subband_one_bit_staged(L, ctx):
    fil = synth.make_1bit(96, 1 << 15, 2.5e-4, 1230.0, 1518.0,
                          [synth.Pulsar(0.02, 100.0, 0.05, 0.1)], seed=4)
    stages = synth.stages_from_table([(0.0, 100.0, 5.0, 1), (100.0, 300.0, 10.0, 2), (300.0, 500.0, 25.0, 4)], True)
    _check(L, ctx, fil, stages, (12, 10))


def test_subband_full_size_sampled(L, ctx):
    # the drift-scan file (256 ch x 2^18, 1001 trials), the two-stage plan the
    # benchmark times; trials at group and launch-batch edges checked exactly
    wl = synth.workload_driftscan()
    _check(L, ctx, wl.fil, wl.stages, (16, 16), trials={0, 1, 15, 16, 255, 256, 500, 511, 512, 999, 1000})


def test_search_on_subband_plan_matches_oracle(L, ctx, small, monkeypatch):
    fil = small.fil
    cfg = L.cfg_of(small.cfg)
    sub = (8, 8)
    plan = L.Plan(L.FilDesc.of(fil), small.stages, subband=sub)
    op = OP.Plan.for_file(fil, small.stages, sub)
    x = OD.channel_major(fil.data, fil.nchan, 8)
    raw = L.pss_search_raw(ctx, plan, _dev(fil.data), cfg, 0, plan.ndm)
    tot = 0
    for i in range(0, plan.ndm, 7):
        _, _, pl = oracle_plane(x, op, i, small.cfg)
        g, r, e = compare_candidates(raw, pl, i, small.cfg.numharm, 0, op.t_span(i), small.cfg.f_lo_hz,
                                     small.cfg.sigma_thr)
        tot += r
    assert tot > 50
    cands = L.pss_search_dm_batch(ctx, plan, _dev(fil.data), cfg, 0, plan.ndm)
    best = cands[np.argmax(cands["sigma"])]
    assert abs(best["dm"] - 50.0) <= 1.0
    # the same search through a prepared batch (graph, default launch shapes) gives the same list
    monkeypatch.setenv("PSS_AUTOTUNE", "0")
    b = L.pss_batch_create(plan, cfg)
    try:
        again = b.run(_dev(fil.data))
    finally:
        b.close()
    assert again.tobytes() == cands.tobytes()


def test_noalloc_refuses_subband_plan(L, small):
    plan = L.Plan(L.FilDesc.of(small.fil), small.stages, subband=(8, 8))
    with pytest.raises(L.PssError) as e:
        L.pss_dedisperse_noalloc(plan, _dev(small.fil.data), 0, 4)
    assert e.value.status == L.PSS_EINVAL


def test_server_serves_subband_plans(L, small, monkeypatch):
    # a two-stage request and an exact one of the same file, served together:
    # each equals its own prepared batch (default launch shapes)
    monkeypatch.setenv("PSS_AUTOTUNE", "0")
    fil, cfg = small.fil, L.cfg_of(small.cfg)
    desc = L.FilDesc.of(fil)
    refs = {}
    for sub in (None, (8, 8)):
        b = L.pss_batch_create(L.Plan(desc, small.stages, subband=sub), cfg)
        refs[sub] = b.run(fil.data)
        b.close()
    srv = L.Server(8 << 30, max_slots=2)
    try:
        tickets = {sub: srv.submit(desc, fil.data, small.stages, cfg, subband=sub) for sub in (None, (8, 8))}
        for sub, t in tickets.items():
            got, _ = srv.poll(t)
            assert got.tobytes() == refs[sub].tobytes(), sub
        with pytest.raises(L.PssError):
            srv.submit(desc, fil.data, small.stages, cfg, subband=(0, 8))
    finally:
        srv.close()
