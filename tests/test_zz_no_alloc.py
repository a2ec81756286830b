"""The allocation-free dedispersion entry point.

pss_dedisperse_noalloc serves callers that cannot allocate device memory
during a call (a real-time ingest thread must not call cudaMalloc, which can
stall the device; a process whose device memory is fully reserved by another
allocator has none to give).  It keeps its scratch in a static device array
shared by all calls.  This file is collected last so that a run stopping at
the first failure has run every other test; it also passes alone in a fresh
process.  The check: two calls in a row through the C ABI give exactly the
int32 series of pss_dedisperse (integer results are compared bit-exactly,
the tolerance every dedispersion test here uses)."""
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


def _noalloc_c(L, plan, dev, b, e, out, stream=None):
    return L.lib().pss_dedisperse_noalloc(plan.h, C.byref(plan.desc.c), C.c_void_p(dev.data_ptr()), b, e,
                                          C.c_void_p(out.data_ptr()), stream)


def test_noalloc_matches_pss_dedisperse_twice(L):
    import torch
    ctx = L.Context(0)
    # two different files and DM ranges, one call right after the other
    cases = []
    wl = synth.workload_small()
    cases.append((wl.fil, wl.stages, (0, 101)))
    fil2 = synth.make_1bit(96, 1 << 15, 2.5e-4, 1230.0, 1518.0, [synth.Pulsar(0.02, 100.0, 0.05, 0.1)], seed=4)
    st2 = synth.stages_from_table([(0.0, 100.0, 5.0, 1), (100.0, 300.0, 10.0, 2)], True)
    cases.append((fil2, st2, (7, 33)))
    for fil, stages, (b, e) in cases:
        plan = L.Plan(L.FilDesc.of(fil), stages)
        dev = torch.from_numpy(fil.data).cuda()
        ref = L.pss_dedisperse(ctx, plan, dev, b, e).cpu().numpy()
        total = ref.shape[0]
        out = torch.full((total,), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        st = _noalloc_c(L, plan, dev, b, e, out)
        assert st == L.PSS_OK, L.lib().pss_last_error().decode()
        np.testing.assert_array_equal(out.cpu().numpy(), ref)
    ctx.close()


def test_noalloc_rejects_oversized_request(L):
    import torch
    fil = synth.make_8bit(256, 1 << 18, 2e-4, 1050.0, 1450.0, [], seed=2)
    plan = L.Plan(L.FilDesc.of(fil), [synth.Stage(0.0, 1.0, 4, 1)])
    dev = torch.from_numpy(fil.data).cuda()
    out = torch.empty(4 * plan.trial(0)["nv"], dtype=torch.int32, device="cuda")
    st = _noalloc_c(L, plan, dev, 0, 4, out)
    assert st == L.PSS_EINVAL
    assert "scratch" in L.lib().pss_last_error().decode()
