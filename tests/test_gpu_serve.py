"""Batched (graph-captured) search and the request loop, through the C ABI.

A file's candidates do not depend on how it was run: a prepared batch, the
plain pss_search_dm_batch call, and the server with other files of other
shapes in flight all give the same bytes."""
import numpy as np
import pytest

from paper_1912_12807_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def untuned(monkeypatch):
    # byte-for-byte comparisons with the untuned plain call: keep the default
    # launch shapes (the tuned FFT split changes FP32 rounding only)
    monkeypatch.setenv("PSS_AUTOTUNE", "0")


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


def _case_a(seed=1001):
    return synth.workload_small(seed=seed, nsamp=1 << 15)


def _case_b():
    # another shape: 32 channels, 2^14 samples, an acceleration search
    fil = synth.make_8bit(32, 1 << 14, 2e-4, 1200.0, 1500.0,
                          [synth.Pulsar(0.01, 20.0, 0.05, 0.6, z_direct=6.0)], seed=77)
    return synth.Workload("b", fil, [synth.Stage(0.0, 2.0, 31, 1)],
                          synth.SearchCfg(zmax=20, dz=2.0, numharm=4, whiten_block=256))


def _alone(L, ctx, wl):
    desc = L.FilDesc.of(wl.fil)
    plan = L.Plan(desc, wl.stages)
    return L.pss_search_dm_batch(ctx, plan, wl.fil.data, L.cfg_of(wl.cfg), 0, plan.ndm)


def _same(a, b):
    return a.shape == b.shape and a.tobytes() == b.tobytes()


def test_batch_equals_search_dm_batch(L, ctx):
    import torch
    for wl in (_case_a(), _case_b()):
        ref = _alone(L, ctx, wl)
        assert ref.shape[0] > 0
        plan = L.Plan(L.FilDesc.of(wl.fil), wl.stages)
        cfg = L.cfg_of(wl.cfg)
        b = L.pss_batch_create(plan, cfg)
        assert b.footprint > 0
        assert L.pss_search_footprint(plan, cfg) >= b.footprint
        assert _same(b.run(wl.fil.data), ref)
        assert _same(b.run(wl.fil.data), ref)  # the graph relaunches cleanly
        assert _same(b.run(torch.from_numpy(wl.fil.data).cuda()), ref)
        b.close()


def test_batch_serves_other_files_of_its_shape(L, ctx):
    a1, a2 = _case_a(1001), _case_a(4242)
    plan = L.Plan(L.FilDesc.of(a1.fil), a1.stages)
    b = L.Batch(plan, L.cfg_of(a1.cfg))
    r1, r2 = b.run(a1.fil.data), b.run(a2.fil.data)
    assert _same(r1, _alone(L, ctx, a1)) and _same(r2, _alone(L, ctx, a2))
    assert not _same(r1, r2)
    b.close()


def test_batch_grows_when_detections_overflow(L, ctx):
    # a 0.5-sigma threshold turns most local maxima into detections: more
    # than the batch's initial device capacity of 2^18
    fil = synth.make_8bit(64, 1 << 15, 2e-4, 1200.0, 1500.0, [], seed=9)
    wl = synth.Workload("o", fil, [synth.Stage(0.0, 1.0, 81, 1)],
                        synth.SearchCfg(zmax=0, numharm=1, sigma_thr=0.5, min_dm_hits=1))
    plan = L.Plan(L.FilDesc.of(fil), wl.stages)
    cfg = L.cfg_of(wl.cfg)
    raw = L.pss_search_raw(ctx, plan, fil.data, cfg, 0, plan.ndm)
    assert raw.shape[0] > (1 << 18)
    b = L.Batch(plan, cfg)
    assert _same(b.run(fil.data), _alone(L, ctx, wl))
    b.close()


def test_server_alone_vs_mix_identical(L, ctx):
    a, b, c = _case_a(1001), _case_b(), _case_a(5151)
    ref = {k: _alone(L, ctx, w) for k, w in (("a", a), ("b", b), ("c", c))}
    srv = L.pss_server_create(8 << 30, max_slots=3)
    order = [("a", a), ("b", b), ("c", c), ("a", a), ("b", b), ("c", c), ("a", a)]
    tickets = [(k, srv.submit(L.FilDesc.of(w.fil), w.fil.data, w.stages, L.cfg_of(w.cfg))) for k, w in order]
    for k, t in tickets:
        got, lat = srv.poll(t, timeout_ms=120000)
        assert lat > 0
        assert _same(got, ref[k]), k
    st = srv.stats()
    assert st["completed"] == len(order)
    assert 0 < st["p50_s"] <= st["p99_s"]
    assert 0 < st["bytes_in_use"] <= 8 << 30
    srv.close()


def test_server_tight_budget_admits_one_at_a_time(L, ctx):
    a, b = _case_a(1001), _case_b()
    pa = L.Plan(L.FilDesc.of(a.fil), a.stages)
    pb = L.Plan(L.FilDesc.of(b.fil), b.stages)
    need = max(L.pss_search_footprint(pa, L.cfg_of(a.cfg)), L.pss_search_footprint(pb, L.cfg_of(b.cfg)))
    srv = L.Server(need + need // 4, max_slots=3)
    ref = {"a": _alone(L, ctx, a), "b": _alone(L, ctx, b)}
    ts = [(k, srv.submit(L.FilDesc.of(w.fil), w.fil.data, w.stages, L.cfg_of(w.cfg)))
          for k, w in (("a", a), ("b", b), ("a", a), ("b", b))]
    for k, t in ts:
        got, _ = srv.poll(t, timeout_ms=120000)
        assert _same(got, ref[k])
        assert srv.stats()["bytes_in_use"] <= need + need // 4
    srv.close()


def test_server_budget_too_small_fails_that_file_only(L, ctx):
    a = _case_a(1001)
    srv = L.Server(1 << 20, max_slots=2)
    t = srv.submit(L.FilDesc.of(a.fil), a.fil.data, a.stages, L.cfg_of(a.cfg))
    with pytest.raises(L.PssError) as e:
        srv.poll(t, timeout_ms=60000)
    assert e.value.status == L.PSS_ENOMEM
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_server_poll_states_and_bad_requests(L, ctx):
    a = _case_a(1001)
    srv = L.Server(8 << 30, max_slots=1)
    desc = L.FilDesc.of(a.fil)
    bad = L.cfg_of(a.cfg)
    bad.numharm = 3
    with pytest.raises(L.PssError) as e:
        srv.submit(desc, a.fil.data, a.stages, bad)
    assert e.value.status == L.PSS_EINVAL
    t1 = srv.submit(desc, a.fil.data, a.stages, L.cfg_of(a.cfg))
    t2 = srv.submit(desc, a.fil.data, a.stages, L.cfg_of(a.cfg))
    # one slot: the second file waits for the first (whose batch is still
    # being prepared and captured)
    with pytest.raises(L.PssError) as e:
        srv.poll(t2, timeout_ms=0)
    assert e.value.status == L.PSS_ENOTREADY
    with pytest.raises(L.PssError) as e:
        srv.poll(t2, timeout_ms=1)
    assert e.value.status == L.PSS_ETIMEOUT
    r2, _ = srv.poll(t2, timeout_ms=120000)
    r1, _ = srv.poll(t1, timeout_ms=120000)
    assert _same(r1, r2)
    for t in (t1, 987654):
        with pytest.raises(L.PssError) as e:
            srv.poll(t, timeout_ms=0)
        assert e.value.status == L.PSS_EINVAL
    srv.close()


def test_take_cands_after_ecap_needs_no_second_search(L, ctx):
    import ctypes as C
    a = _case_a(1001)
    ref = _alone(L, ctx, a)
    assert ref.shape[0] > 1
    plan = L.Plan(L.FilDesc.of(a.fil), a.stages)
    cfg = L.cfg_of(a.cfg)
    one = np.zeros(1, dtype=L.CAND_DTYPE)
    n = C.c_int64()
    st = L.lib().pss_search_dm_batch(ctx.h, plan.h, C.byref(plan.desc.c), C.c_void_p(a.fil.data.ctypes.data), 0,
                                     C.byref(cfg), 0, plan.ndm, one.ctypes.data, 1, C.byref(n), None)
    assert st == L.PSS_ECAP and n.value == ref.shape[0]
    out = np.zeros(n.value, dtype=L.CAND_DTYPE)
    assert L.lib().pss_ctx_take_cands(ctx.h, out.ctypes.data, n.value, C.byref(n)) == L.PSS_OK
    assert _same(out, ref)
    b = L.Batch(plan, cfg)
    assert _same(b.run(a.fil.data, cap=1), ref)
    b.close()
    fresh = L.Context(0)
    assert L.lib().pss_ctx_take_cands(fresh.h, out.ctypes.data, n.value, C.byref(n)) == L.PSS_EINVAL
    fresh.close()


def test_alternate_launch_shapes_are_exact(L, ctx, monkeypatch):
    # 16 points per lane in the harmonic sum, a 64 KiB dedispersion chunk budget
    # and the warp-per-block whitening median: the same arithmetic, the same bytes
    for case in (_case_a(1001), _case_b()):
        for pin, form in (("0,16,64,1,0", 1), ("0,8,96,2,0", 2), ("0,8,96,0,0", 0)):
            # the warp-pair (2) and block (0) whitening forms select the same median
            monkeypatch.setenv("PSS_TUNE", pin)
            plan = L.Plan(L.FilDesc.of(case.fil), case.stages)
            b = L.Batch(plan, L.cfg_of(case.cfg))
            assert b.tuning["whiten_form"] == form
            got = b.run(case.fil.data)
            b.close()
            monkeypatch.delenv("PSS_TUNE")
            assert _same(got, _alone(L, ctx, case)), pin
    monkeypatch.setenv("PSS_TUNE", "0,7,64,1")
    with pytest.raises(L.PssError):
        L.Batch(L.Plan(L.FilDesc.of(_case_a().fil), _case_a().stages), L.cfg_of(_case_a().cfg))


def test_autotuned_batch_and_server(L, ctx, monkeypatch):
    monkeypatch.setenv("PSS_AUTOTUNE", "1")
    a, c = _case_a(1001), _case_a(5151)
    plan = L.Plan(L.FilDesc.of(a.fil), a.stages)
    cfg = L.cfg_of(a.cfg)
    b = L.Batch(plan, cfg)
    t = b.tuning
    assert t["harm_run"] in (8, 16) and t["dedisp_kb"] in (64, 96) and t["fft_split"] >= 0
    assert t["whiten_form"] in (0, 1, 2)
    got, ref = b.run(a.fil.data), _alone(L, ctx, a)
    # same detections; powers within the parity tolerance of the untuned search
    key = lambda x: set(zip(x["dm_idx"].tolist(), x["numharm"].tolist(), x["h"].tolist(), x["j"].tolist()))
    assert len(key(got) ^ key(ref)) <= max(2, len(ref) // 50)
    common = {k: p for k, p in zip(zip(ref["dm_idx"].tolist(), ref["numharm"].tolist(), ref["h"].tolist(),
                                       ref["j"].tolist()), ref["power"].tolist())}
    for row in got:
        k = (int(row["dm_idx"]), int(row["numharm"]), int(row["h"]), int(row["j"]))
        if k in common:
            assert abs(row["power"] - common[k]) <= 1e-4 * max(common[k], 1.0)
    b2 = L.Batch(plan, cfg)
    assert b2.tuning == t  # remembered per shape
    b2.close()
    b.close()
    # served: alone and in a mix give the same bytes (one tuning per shape)
    srv = L.Server(8 << 30, max_slots=2)
    desc = L.FilDesc.of(a.fil)
    alone = srv.poll(srv.submit(desc, a.fil.data, a.stages, cfg), 120000)[0]
    ts = [srv.submit(L.FilDesc.of(w.fil), w.fil.data, w.stages, L.cfg_of(w.cfg)) for w in (c, a, _case_b(), a)]
    outs = [srv.poll(t, 120000)[0] for t in ts]
    assert _same(outs[1], alone) and _same(outs[3], alone)
    srv.close()
