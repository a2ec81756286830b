"""GPU single-pulse search (pss_single_pulse) against the oracle
(oracle/single_pulse.py) on the same dedispersed series: the pruned event
lists are identical (trial, start, width, boxcar sum) and the S/N agrees to
FP64 rounding."""
import numpy as np
import pytest

from oracle import dedisperse as OD
from oracle import plan as OP
from oracle import single_pulse as OSP
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


def _bursty(nchan=64, nsamp=1 << 15, seed=11):
    # a long-period pulsar (a few bright, wide single pulses) and a short-period one
    return synth.make_8bit(nchan, nsamp, 2e-4, 1200.0, 1500.0,
                           [synth.Pulsar(1.3, 45.0, 0.004, 3.0, phase0=0.3),
                            synth.Pulsar(0.0333, 20.0, 0.05, 0.3)], seed=seed)


def _compare(L, ctx, fil, stages, widths, thr, sub=None, mask=None, rng_=None):
    desc = L.FilDesc.of(fil, chan_mask=mask)
    plan = L.Plan(desc, stages, subband=sub)
    op = OP.Plan.for_file(fil, stages, sub)
    x = OD.channel_major(fil.data, fil.nchan, fil.nbits)
    b, e = rng_ if rng_ else (0, plan.ndm)
    got = L.pss_single_pulse(ctx, plan, _dev(fil.data), b, e, widths=widths, sigma_thr=thr)
    ref = []
    for i in range(b, e):
        ds = int(op.ds_of[i])
        if sub is None:
            s = OD.dedisperse(x, op.delays[i], op.max_delay, ds, mask)
        else:
            s = OSB.dedisperse_subband(x, op.sub, i, op.max_delay, ds, mask)
        ref += [(i, t, w, B, sn) for t, w, B, sn in OSP.search_series(s, widths, thr)]
    assert len(got) == len(ref)
    for g, r in zip(got, ref):
        assert (int(g["dm_idx"]), int(g["t"]), int(g["width"]), int(g["boxsum"])) == r[:4]
        assert abs(float(g["snr"]) - r[4]) <= 1e-12 * abs(r[4])
    return got


def test_single_pulse_matches_oracle(L, ctx):
    fil = _bursty()
    stages = [synth.Stage(30.0, 1.0, 31, 1), synth.Stage(61.0, 2.0, 5, 2)]
    got = _compare(L, ctx, fil, stages, L.SP_WIDTHS, 6.0)
    # the bright pulses are found at the pulsar's DM with a width near their own
    top = got[np.argmax(got["snr"])]
    assert abs(float(top["dm_idx"]) - 15) <= 2   # DM 45 is trial 15 of the first stage


def test_single_pulse_low_threshold_many_events(L, ctx):
    # a low threshold gives many noise events: exercises the local-maximum
    # windows, the pruning and the event buffer
    fil = _bursty(seed=12)
    stages = [synth.Stage(0.0, 3.0, 9, 1)]
    got = _compare(L, ctx, fil, stages, (1, 3, 8, 30, 200, 1024), 3.0)
    assert len(got) > 100


def test_single_pulse_two_stage_plan_mask_downsampled(L, ctx):
    fil = _bursty(seed=13)
    mask = np.ones(64, dtype=np.uint8)
    mask[[2, 9, 33]] = 0
    stages = [synth.Stage(20.0, 2.0, 12, 2), synth.Stage(44.0, 4.0, 6, 8)]
    _compare(L, ctx, fil, stages, (1, 2, 4, 16, 64), 5.0, sub=(8, 4), mask=mask, rng_=(3, 17))


def test_single_pulse_constant_input_and_errors(L, ctx):
    fil = _bursty(nsamp=1 << 13)
    fil.data[:] = 128
    plan = L.Plan(L.FilDesc.of(fil), [synth.Stage(0.0, 5.0, 4, 1)])
    assert len(L.pss_single_pulse(ctx, plan, _dev(fil.data), 0, 4, sigma_thr=1.0)) == 0
    with pytest.raises(L.PssError) as e:
        L.pss_single_pulse(ctx, plan, _dev(fil.data), 0, 4, widths=(0, 4))
    assert e.value.status == L.PSS_EINVAL
    with pytest.raises(L.PssError):
        L.pss_single_pulse(ctx, plan, _dev(fil.data), 0, 4, widths=(2048,))
    with pytest.raises(L.PssError):
        L.pss_single_pulse(ctx, plan, _dev(fil.data), 0, 4, widths=tuple(range(1, 40)))


def test_single_pulse_wide_sums(L, ctx):
    # heavy downsampling: window sums beyond 32 bits, the 64-bit prefix form
    fil = _bursty(nsamp=1 << 17, seed=14)
    stages = [synth.Stage(20.0, 5.0, 6, 256)]
    _compare(L, ctx, fil, stages, (1, 2, 4, 16), 3.0)
