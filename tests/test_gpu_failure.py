"""Failure detection without a GPU fault, through the C ABI.

* A staging-barrier wait that runs out: a context whose dedispersion data
  waits give up after one non-blocking poll (pss_ctx_set_wait_limit) makes
  the kernels set the error flag, drain their bulk copies in flight and
  leave; the calls return PSS_ETIMEOUT (the asynchronous pss_dedisperse
  through pss_ctx_check), and after the limit is restored the same context
  gives the oracle's bytes.  Exact and two-stage plans.
* A device allocation that fails (pss_debug_fail_alloc): the call returns
  PSS_ENOMEM, device memory is not leaked, and the next call succeeds.
* A request whose worker meets such a failure in the request loop fails
  alone: the other tickets complete with the bytes of a search alone."""
import numpy as np
import pytest

from oracle import dedisperse as OD
from oracle import plan as OP
from paper_1912_12807_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1912_12807_gb300 import pss
    pss.lib()
    return pss


@pytest.fixture(scope="module")
def small():
    return synth.workload_small()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_wait_runs_out_then_context_recovers(L, small):
    fil = small.fil
    plan = L.Plan(L.FilDesc.of(fil), small.stages)
    cfg = L.cfg_of(small.cfg)
    dev = _dev(fil.data)
    ctx = L.Context(0)
    try:
        ref = L.pss_search_dm_batch(ctx, plan, dev, cfg, 0, plan.ndm).tobytes()
        L.pss_ctx_set_wait_limit(ctx, 1)
        with pytest.raises(L.PssError) as ei:
            L.pss_search_dm_batch(ctx, plan, dev, cfg, 0, plan.ndm)
        assert ei.value.status == L.PSS_ETIMEOUT
        L.pss_dedisperse(ctx, plan, dev, 0, plan.ndm)
        with pytest.raises(L.PssError) as ei:
            L.pss_ctx_check(ctx)
        assert ei.value.status == L.PSS_ETIMEOUT
        L.pss_ctx_check(ctx)  # reported once, then clear
        # the two-stage scheme's stage-2 kernel has the same bounded waits
        sub = L.Plan(L.FilDesc.of(fil), small.stages, subband=(8, 8))
        with pytest.raises(L.PssError) as ei:
            L.pss_search_dm_batch(ctx, sub, dev, cfg, 0, sub.ndm)
        assert ei.value.status == L.PSS_ETIMEOUT
        # restored: the same context gives the oracle's series and the same candidates
        L.pss_ctx_set_wait_limit(ctx, 0)
        out = L.pss_dedisperse(ctx, plan, dev, 0, plan.ndm).cpu().numpy()
        L.pss_ctx_check(ctx)
        op = OP.Plan.for_file(fil, small.stages)
        x = OD.channel_major(fil.data, fil.nchan, 8)
        nv = op.nv_nfft(0)[0]
        for i in (0, 50, 100):
            np.testing.assert_array_equal(out[i * nv:(i + 1) * nv], OD.dedisperse(x, op.delays[i], op.max_delay, 1))
        assert L.pss_search_dm_batch(ctx, plan, dev, cfg, 0, plan.ndm).tobytes() == ref
        with pytest.raises(L.PssError):
            L.pss_ctx_set_wait_limit(ctx, -1)
    finally:
        ctx.close()


def test_allocation_failure_returns_enomem_without_leaks(L, small):
    import torch
    fil = small.fil
    plan = L.Plan(L.FilDesc.of(fil), small.stages)
    cfg = L.cfg_of(small.cfg)
    ref_ctx = L.Context(0)
    ref = L.pss_search_dm_batch(ref_ctx, plan, fil.data, cfg, 0, plan.ndm).tobytes()
    ref_ctx.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    try:
        for n in range(1, 12):
            ctx = L.Context(0)
            L.pss_debug_fail_alloc(n)
            try:
                got = L.pss_search_dm_batch(ctx, plan, fil.data, cfg, 0, plan.ndm).tobytes()
                assert got == ref  # the refused allocation came after this search's last one
            except L.PssError as e:
                assert e.status == L.PSS_ENOMEM, e
                failures += 1
                L.pss_debug_fail_alloc(0)
                # the same context recovers
                assert L.pss_search_dm_batch(ctx, plan, fil.data, cfg, 0, plan.ndm).tobytes() == ref
            finally:
                L.pss_debug_fail_alloc(0)
                ctx.close()
    finally:
        L.pss_debug_fail_alloc(0)
    assert failures >= 5
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 >= free0 - (64 << 20), (free0, free1)


def test_server_request_failure_is_isolated(L, small):
    fil = small.fil
    cfg = L.cfg_of(small.cfg)
    stages = small.stages
    others = [synth.make_8bit(64, 1 << 15, 2e-4, 1200.0, 1500.0, [synth.Pulsar(0.02 + 0.01 * k, 40.0, 0.05, 0.6)],
                              seed=70 + k) for k in range(3)]
    # what each file gives alone: a prepared batch (the per-shape slots, autotuned) and a
    # default context (the grouped slots)
    refs = {1: [], 4: []}
    for f in others:
        p = L.Plan(L.FilDesc.of(f), stages)
        b = L.Batch(p, cfg)
        refs[1].append(b.run(f.data).tobytes())
        b.close()
        ctx = L.Context(0)
        refs[4].append(L.pss_search_dm_batch(ctx, p, f.data, cfg, 0, p.ndm).tobytes())
        ctx.close()
    for group in (1, 4):
        srv = L.Server(16 << 30, max_slots=1, max_group=group)
        try:
            # the first request's preparation meets a refused allocation; the queue behind it is served
            L.pss_debug_fail_alloc(2)
            t_bad = srv.submit(L.FilDesc.of(fil), fil.data, stages, cfg)
            with pytest.raises(L.PssError) as ei:
                srv.poll(t_bad)
            assert ei.value.status == L.PSS_ENOMEM
            L.pss_debug_fail_alloc(0)
            ts = [srv.submit(L.FilDesc.of(f), f.data, stages, cfg) for f in others]
            assert [srv.poll(t)[0].tobytes() for t in ts] == refs[group]
        finally:
            L.pss_debug_fail_alloc(0)
            srv.close()
