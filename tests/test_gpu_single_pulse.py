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


def _tie_file(spikes, seed, N=8192, nchan=64, base=100):
    # Channel 0 carries base + x[t], the other channels base: at DM 0 the
    # trial's series is nchan*base + x[t].  x is +-2 noise plus the given
    # samples, with sum 0 and square sum 4N, so mu = nchan*base and sigma = 2
    # come out exactly in FP64 and the ties below are exact.
    rng = np.random.default_rng(seed)
    x = np.zeros(N, np.int64)
    tot = (4 * N - sum(v * v for v in spikes.values())) // 4
    diff = -sum(spikes.values()) // 2
    n_plus = (tot + diff) // 2
    pos = rng.permutation(np.array([t for t in range(N) if t not in spikes]))
    x[pos[:n_plus]] = 2
    x[pos[n_plus:tot]] = -2
    for t, v in spikes.items():
        x[t] = v
    assert x.sum() == 0 and (x * x).sum() == 4 * N
    data = np.full((N, nchan), base, np.uint8)
    data[:, 0] = base + x
    fch0, foff = synth.band(1200.0, 1500.0, nchan)
    return synth.Filterbank(nchan, N, 2e-4, fch0, foff, 8, data, [])


def test_single_pulse_exact_ties(L, ctx):
    stages = [synth.Stage(0.0, 1.0, 1, 1)]
    # a one-sample boxcar exactly at 5 sigma (6400 + 10) is an event; a threshold
    # 1e-9 sigma higher (a threshold above 6410 after rounding) leaves none
    fil = _tie_file({4000: 10}, 7)
    got = _compare(L, ctx, fil, stages, (1,), 5.0)
    assert [(int(g["t"]), int(g["width"]), int(g["boxsum"])) for g in got] == [(4000, 1, 6410)]
    assert len(_compare(L, ctx, fil, stages, (1,), 5.0 + 1e-9)) == 0
    # three equal samples make two equal two-sample boxcars: one event, at the first
    fil = _tie_file({3000: 10, 3001: 10, 3002: 10}, 8)
    got = _compare(L, ctx, fil, stages, (2,), 4.0)
    assert [(int(g["t"]), int(g["width"])) for g in got] == [(3000, 2)]
    # 4, 8, 4 between zeros: the one-sample boxcar 8 and the four-sample boxcar 16
    # have the same S/N 4; they overlap and the narrower one is kept
    fil = _tie_file({4998: 0, 4999: 0, 5000: 4, 5001: 8, 5002: 4, 5003: 0, 5004: 0}, 9)
    got = _compare(L, ctx, fil, stages, (1, 4), 3.0)
    assert [(int(g["t"]), int(g["width"]), float(g["snr"])) for g in got] == [(5001, 1, 4.0)]
