"""Several files in one launch per stage (pss_search_multi) and the grouped
request loop (pss_server_create_grouped), through the C ABI.

A group mixes channel counts (64 to 300: both dedispersion kernel
variants), sample counts, 8-bit and 1-bit files, channel-major layout, a
channel mask and staged plans with downsampled rows (several transform
lengths in one group).  Every file's sorted, sifted candidate list must be
byte-identical to that file searched alone with pss_search_dm_batch (whose
output is compared with the oracle in the other GPU tests): eagerly (the
first group on a context), as a captured graph (later groups), with host or
device input, at zmax 0 and zmax > 0, and served in groups."""
import ctypes as C

import numpy as np
import pytest

from paper_1912_12807_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1912_12807_gb300 import pss
    pss.lib()
    return pss


def _group(L):
    """[(desc, data, stages)] of five files of different shapes."""
    out = []
    small = synth.workload_small(nsamp=1 << 15)
    out.append((L.FilDesc.of(small.fil), small.fil.data, [synth.Stage(20.0, 1.0, 61, 1)]))
    f2 = synth.make_8bit(128, (1 << 16) + 777, 2e-4, 1100.0, 1400.0, [synth.Pulsar(0.0121, 42.0, 0.05, 0.6)],
                         seed=21)
    out.append((L.FilDesc.of(f2), f2.data, [synth.Stage(0.0, 2.0, 40, 1)]))
    f3 = synth.make_1bit(96, (1 << 16) + 500, 2.5e-4, 1230.0, 1518.0, [synth.Pulsar(0.02, 100.0, 0.05, 0.1)],
                         seed=4)
    st3 = synth.stages_from_table([(0.0, 100.0, 5.0, 1), (100.0, 300.0, 10.0, 2), (300.0, 500.0, 25.0, 4)], True)
    out.append((L.FilDesc.of(f3), f3.data, st3))
    f4 = synth.make_8bit(300, 40000, 2e-4, 1200.0, 1500.0, [synth.Pulsar(0.05, 30.0, 0.05, 0.8)], seed=300)
    out.append((L.FilDesc.of(f4), f4.data, [synth.Stage(0.0, 3.0, 20, 1), synth.Stage(60.0, 5.0, 10, 2)]))
    mask = np.ones(64, dtype=np.uint8)
    mask[[0, 7, 8, 40, 63]] = 0
    cm = np.ascontiguousarray(small.fil.data.T)
    out.append((L.FilDesc.of(small.fil, chan_mask=mask, layout=1), cm, [synth.Stage(30.0, 1.0, 41, 1)]))
    return out


def _alone(L, files, cfg):
    res = []
    for desc, data, stages in files:
        ctx = L.Context(0)
        plan = L.Plan(desc, stages)
        res.append(L.pss_search_dm_batch(ctx, plan, data, cfg, 0, plan.ndm).tobytes())
        ctx.close()
    return res


@pytest.fixture(scope="module")
def group(L):
    return _group(L)


@pytest.mark.parametrize("zmax", [0, 12])
def test_multi_equals_alone(L, group, zmax):
    import torch
    cfg = L.search_cfg(zmax=zmax, dz=2.0, numharm=8)
    ref = _alone(L, group, cfg)
    assert sum(len(r) for r in ref) > 0
    plans = [L.Plan(d, st) for d, _, st in group]
    ctx = L.Context(0)
    try:
        for rep in range(3):  # eager first, then captured graphs
            got = L.pss_search_multi(ctx, cfg, [(p, data) for p, (_, data, _) in zip(plans, group)])
            assert [g.tobytes() for g in got] == ref, "repetition %d" % rep
        dev = [torch.from_numpy(np.ascontiguousarray(data)).cuda() for _, data, _ in group]
        got = L.pss_search_multi(ctx, cfg, [(p, d) for p, d in zip(plans, dev)])
        assert [g.tobytes() for g in got] == ref
        # a different grouping of the same files on the same context
        got = L.pss_search_multi(ctx, cfg, [(plans[k], group[k][1]) for k in (3, 1)])
        assert [g.tobytes() for g in got] == [ref[3], ref[1]]
    finally:
        ctx.close()


def test_multi_capacity_and_errors(L, group):
    cfg = L.search_cfg(zmax=0, numharm=8)
    ref = _alone(L, group, cfg)
    plans = [L.Plan(d, st) for d, _, st in group]
    arr, on_dev, keep = L._multi_files([(p, data) for p, (_, data, _) in zip(plans, group)])
    ctx = L.Context(0)
    try:
        counts = np.zeros(len(group), dtype=np.int64)
        n = C.c_int64()
        out = np.zeros(1, dtype=L.CAND_DTYPE)
        st = L.lib().pss_search_multi(ctx.h, C.byref(cfg), arr, len(group), 0, out.ctypes.data, 1,
                                      counts.ctypes.data, C.byref(n), None)
        assert st == L.PSS_ECAP and n.value == sum(len(r) for r in ref) // L.CAND_DTYPE.itemsize
        assert list(counts) == [len(r) // L.CAND_DTYPE.itemsize for r in ref]
        full = np.zeros(n.value, dtype=L.CAND_DTYPE)
        assert L.lib().pss_ctx_take_cands(ctx.h, full.ctypes.data, n.value, C.byref(n)) == 0
        assert full.tobytes() == b"".join(ref)
        # a two-stage plan is refused; so is an empty group
        sub = L.Plan(group[0][0], group[0][2], subband=(8, 4))
        with pytest.raises(L.PssError):
            L.pss_search_multi(ctx, cfg, [(plans[1], group[1][1]), (sub, group[0][1])])
        with pytest.raises(L.PssError):
            L.pss_search_multi(ctx, cfg, [])
        # host and device inputs are not mixed
        import torch
        with pytest.raises(ValueError):
            L.pss_search_multi(ctx, cfg, [(plans[0], group[0][1]), (plans[1], torch.from_numpy(group[1][1]).cuda())])
        assert L.pss_search_multi_footprint(cfg, [(p, None) for p in plans]) > sum(
            int(np.asarray(d).nbytes) for _, d, _ in group)
    finally:
        ctx.close()


def test_grouped_server_equals_alone(L, group):
    cfg = L.search_cfg(zmax=0, numharm=8)
    ref = _alone(L, group, cfg)
    srv = L.Server(32 << 30, max_slots=1, max_group=8)
    try:
        # a two-stage plan among them runs alone, and gives the single-file path's bytes
        d0, data0, st0 = group[0]
        ctx = L.Context(0)
        sub_ref = L.pss_search_dm_batch(ctx, L.Plan(d0, st0, subband=(8, 4)), data0, cfg, 0,
                                        L.Plan(d0, st0).ndm).tobytes()
        ctx.close()
        for rep in range(2):
            ts = [srv.submit(d, data, st, cfg) for d, data, st in group]
            tsub = srv.submit(d0, data0, st0, cfg, subband=(8, 4))
            got = [srv.poll(t)[0].tobytes() for t in ts]
            assert got == ref, "repetition %d" % rep
            assert srv.poll(tsub)[0].tobytes() == sub_ref
        s = srv.stats()
        assert s["completed"] == 2 * (len(group) + 1)
        assert s["grouped_files"] == 2 * (len(group) + 1) and s["groups"] < s["grouped_files"]
    finally:
        srv.close()


def test_grouped_server_budget(L, group):
    cfg = L.search_cfg(zmax=0, numharm=8)
    d, data, st = group[1]
    fp = L.pss_search_multi_footprint(cfg, [(L.Plan(d, st), None)])
    # a budget for one file at a time still serves every file, and a file above the budget fails alone
    srv = L.Server(fp + (64 << 20), max_slots=1, max_group=4)
    try:
        ts = [srv.submit(d, data, st, cfg) for _ in range(3)]
        big = synth.make_8bit(1024, 1 << 17, 2e-4, 1050.0, 1450.0, [], seed=9)
        tb = srv.submit(L.FilDesc.of(big), big.data, [synth.Stage(0.0, 1.0, 501, 1)], cfg)
        res = [srv.poll(t)[0] for t in ts]
        assert res[0].tobytes() == res[1].tobytes() == res[2].tobytes()
        with pytest.raises(L.PssError) as ei:
            srv.poll(tb)
        assert ei.value.status == L.PSS_ENOMEM
    finally:
        srv.close()
