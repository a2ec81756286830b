"""Pins for the refinement objective (oracle/refine.py)."""
import math

import numpy as np
import pytest

from oracle import refine as RF
from oracle import response as R
from paper_1912_12807_gb300 import synth


def _tone_file(nchan, nsamp, r0, amp=40.0, seed=0):
    # every channel carries the same undispersed tone at r0 bins of the span
    rng = np.random.default_rng(seed)
    t = np.arange(nsamp)
    x = 128 + amp * np.cos(2 * np.pi * r0 * t / nsamp)[:, None] + rng.normal(0, 2.0, (nsamp, nchan))
    data = np.clip(np.rint(x), 0, 255).astype(np.uint8)
    fch0, foff = synth.band(1200.0, 1500.0, nchan)
    return synth.Filterbank(nchan, nsamp, 2e-4, fch0, foff, 8, data, [])


def test_rho_closed_form_matches_quadrature():
    for q in (0.0, 0.5, -2.25, 7.0):
        assert abs(R.rho(q, 0.0) - R.rho_quad(q, 0.0)) < 1e-13
    assert R.rho(1.5, 3.0) == R.rho_quad(1.5, 3.0)


def test_single_channel_peak_and_zero_gradient_at_tone():
    # One channel, one undispersed tone at a half-integer bin r0 of the span:
    # the 2m taps around r0 are symmetric about it, so the objective is
    # (up to the tone's negative-frequency image and 8-bit rounding) even in
    # r - r0: its maximum is at r0 and its slope there vanishes.
    nsamp = 4096
    r0 = 300.5
    fil = _tone_file(1, nsamp, r0, amp=60.0, seed=1)
    fil.data[:] = np.clip(np.rint(128 + 60.0 * np.cos(2 * np.pi * r0 * np.arange(nsamp) / nsamp)),
                          0, 255).astype(np.uint8)[:, None]
    cfg = synth.SearchCfg(zmax=0, numharm=1, whiten_block=64)
    obj = RF.Objective(fil, [synth.Stage(0.0, 1.0, 3, 1)], cfg, dm_idx=0)
    assert obj.nfft == nsamp and obj.nv == nsamp
    best = obj.grid_max(0.0, r0, 0.0, 1, 1.0, 0.0)
    assert abs(best[2] - r0) < 1e-9
    h = 1e-3
    g = (obj(0.0, r0 + h, 0.0, 1) - obj(0.0, r0 - h, 0.0, 1)) / (2 * h)
    d = 0.05
    curv = (obj(0.0, r0 + d, 0.0, 1) - 2 * obj(0.0, r0, 0.0, 1) + obj(0.0, r0 - d, 0.0, 1)) / d ** 2
    assert curv < 0
    assert abs(g) < 1e-2 * abs(curv)


def test_dm_phase_adds_a_delayed_tone_coherently():
    # 32 channels carry one tone at an integer bin r0 of the span, each delayed by the continuous
    # dispersion delay of DM0 (shift theorem: channel c's bin r0 turns by exp(-2 pi i r0 tau_c / T)).
    # At z = 0 and an integer bin the response is a delta, so P_1(DM) / P_1(DM0) must be the array
    # factor |sum_c exp(2 pi i r0 (DM - DM0) dtau_c / T)|^2 / C^2: 1 at DM0 (the phase undoes the
    # delays), falling off on either side; a sign or scale error in the phase moves the peak.
    nchan, nsamp, r0, dm0, tsamp = 32, 4096, 1000, 30.0, 2e-4
    fch0, foff = synth.band(1200.0, 1500.0, nchan)
    cfg = synth.SearchCfg(zmax=0, numharm=1, whiten_block=64)
    stages = [synth.Stage(0.0, 1e-4, 2, 1)]  # delays that round to 0 samples: N_v = nfft = nsamp
    zero = synth.Filterbank(nchan, nsamp, tsamp, fch0, foff, 8, np.zeros((nsamp, nchan), np.uint8), [])
    dtau = RF.Objective(zero, stages, cfg, dm_idx=0).dtau  # seconds of delay per unit DM, per channel
    T = nsamp * tsamp
    t = np.arange(nsamp)[:, None] * tsamp
    # seeded noise keeps the whitening block medians above 0 (the rounding error of the tone alone
    # repeats every 512 samples and leaves most bins of a block empty)
    noise = np.random.default_rng(5).normal(0.0, 2.0, (nsamp, nchan))
    x = 128 + 100 * np.cos(2 * np.pi * r0 * (t - dm0 * dtau[None, :]) / T) + noise
    fil = synth.Filterbank(nchan, nsamp, tsamp, fch0, foff, 8, np.clip(np.rint(x), 0, 255).astype(np.uint8), [])
    obj = RF.Objective(fil, stages, cfg, dm_idx=0)
    assert obj.nv == obj.nfft == nsamp and abs(obj.T - T) < 1e-12
    peak = obj(dm0, float(r0), 0.0, 1)
    for ddm in (0.05, -0.05, 0.2, -0.3, 0.5, 2 * dm0):
        af = abs(np.sum(np.exp(2j * np.pi * r0 * ddm * dtau / T))) ** 2 / nchan ** 2
        assert abs(obj(dm0 + ddm, float(r0), 0.0, 1) / peak - af) < 1e-3, ddm
    assert obj(-dm0, float(r0), 0.0, 1) < 0.05 * peak


def test_dispersed_pulsar_prefers_its_dm():
    wl = synth.workload_small(nsamp=1 << 14)
    obj = RF.Objective(wl.fil, [synth.Stage(40.0, 1.0, 21, 1)], wl.cfg, dm_idx=10)
    r = (1 / 0.0333) * obj.T  # fundamental of the injected 33.3 ms pulsar
    at = max(obj(50.0, r + d, 0.0, 8) for d in np.arange(-1, 1.01, 0.125))
    off = max(obj(20.0, r + d, 0.0, 8) for d in np.arange(-1, 1.01, 0.125))
    assert at > 4 * off


def _noisy_chirp_file(nchan, nsamp, seed):
    # noise plus a drifting tone (r = 700.3 -> 712.3 bins over the span) in every channel
    rng = np.random.default_rng(seed)
    u = np.arange(nsamp) / nsamp
    tone = 30.0 * np.cos(2 * np.pi * (700.3 * u + 6.0 * u * u))
    x = 128 + tone[:, None] + rng.normal(0, 6.0, (nsamp, nchan))
    fch0, foff = synth.band(1200.0, 1500.0, nchan)
    return synth.Filterbank(nchan, nsamp, 2e-4, fch0, foff, 8, np.clip(np.rint(x), 0, 255).astype(np.uint8), [])


@pytest.mark.parametrize("ds", [1, 2])
def test_one_channel_without_dispersion_is_the_search_plane(ds):
    # One channel is its own reference frequency, so every delay and every DM
    # phase vanishes: the channel's spectrum is the trial's spectrum, and
    # g |sum_q A_q conj(rho)|^2 / E equals the plane value |sum_q A'_q conj(rho)|^2 / E
    # of the whitened spectrum A' = sqrt(g) A wherever the taps stay inside one
    # whitening block.  So P_h(DM, r, z) = sum_k plane(k z)[2 k r] at any DM,
    # the sum over harmonics taking harmonic k at (k r, k z) in its own block.
    from oracle import search as S
    nsamp = 1 << 13
    fil = _noisy_chirp_file(1, nsamp, 3)
    cfg = synth.SearchCfg(zmax=0, numharm=2, whiten_block=256)
    stages = [synth.Stage(0.0, 1.0, 2, ds)]
    obj = RF.Objective(fil, stages, cfg, dm_idx=0)
    assert not obj.dtau.any()
    x_cm = np.ascontiguousarray(fil.data.T)
    _, Ap = S.spectrum_of_trial(x_cm, obj.P, 0, cfg.whiten_block)
    rows = {}

    def plane(z, h):
        if z not in rows:
            rows[z] = R.plane_row_direct(Ap, z, cfg.halfwidth_extra)
        return rows[z][h]

    # fundamentals on the half-bin grid whose taps, and harmonic 2's, stay inside one
    # 256-bin block (block 0 near DC, where taps fall below bin 0, included; 706 is on the chirp)
    for r, z in ((3.0, 0.0), (2.5, 6.0), (175.0, 0.0), (175.5, 6.0), (90.5, -8.0), (300.0, 3.0), (706.0, 12.0)):
        h = int(2 * r)
        want1 = plane(z, h)
        want2 = want1 + plane(2 * z, 2 * h)
        for dm in (0.0, 37.0):
            assert abs(obj(dm, r, z, 1) - want1) <= 1e-9 * want1, (r, z)
            assert abs(obj(dm, r, z, 2) - want2) <= 1e-9 * want2, (r, z)


def test_dm_phase_uses_the_plans_delays():
    # the continuous delay the objective undoes is the plan's unrounded delay
    # (pinned to the cold-plasma sweep in the plan tests), in seconds
    fil = _noisy_chirp_file(16, 2048, 4)
    cfg = synth.SearchCfg(zmax=0, numharm=1, whiten_block=64)
    stages = [synth.Stage(0.0, 10.0, 5, 1)]
    obj = RF.Objective(fil, stages, cfg, dm_idx=0)
    from oracle import plan as P
    for dm in (10.0, 40.0):
        v = P.delay_values(np.array([dm]), obj.P.freqs, fil.tsamp_s)[0]
        np.testing.assert_allclose(dm * obj.dtau / fil.tsamp_s, v, rtol=1e-13, atol=1e-12)


def test_harmonic_k_turns_by_k_times_the_phase():
    # A tone at r0 and its second harmonic at 2 r0, both delayed channel by
    # channel by DM0: harmonic 2 of the fundamental r0 realigns at DM0 and
    # falls off as the array factor at 2 r0, |sum_c exp(2 pi i 2 r0 dDM dtau_c / T)|^2 / C^2.
    nchan, nsamp, r0, dm0, tsamp = 16, 4096, 500, 20.0, 2e-4
    fch0, foff = synth.band(1200.0, 1500.0, nchan)
    cfg = synth.SearchCfg(zmax=0, numharm=2, whiten_block=64)
    stages = [synth.Stage(0.0, 1e-4, 2, 1)]
    zero = synth.Filterbank(nchan, nsamp, tsamp, fch0, foff, 8, np.zeros((nsamp, nchan), np.uint8), [])
    dtau = RF.Objective(zero, stages, cfg, dm_idx=0).dtau
    T = nsamp * tsamp
    t = np.arange(nsamp)[:, None] * tsamp - dm0 * dtau[None, :]
    x = 128 + 50 * np.cos(2 * np.pi * r0 * t / T) + 50 * np.cos(2 * np.pi * 2 * r0 * t / T)
    x = x + np.random.default_rng(6).normal(0.0, 2.0, (nsamp, nchan))
    fil = synth.Filterbank(nchan, nsamp, tsamp, fch0, foff, 8, np.clip(np.rint(x), 0, 255).astype(np.uint8), [])
    obj = RF.Objective(fil, stages, cfg, dm_idx=0)
    peak = obj.harmonic(dm0, float(r0), 0.0, 2)
    for ddm in (0.05, -0.1, 0.25):
        af = abs(np.sum(np.exp(2j * np.pi * 2 * r0 * ddm * dtau / T))) ** 2 / nchan ** 2
        assert abs(obj.harmonic(dm0 + ddm, float(r0), 0.0, 2) / peak - af) < 2e-3, ddm


def test_grid_reaches_both_ends_of_the_cell():
    # the fine grid spans +-1 bin inclusive: a tone one bin above the start
    # is found at the grid's last r point
    nsamp, r0 = 4096, 300.5
    fil = _tone_file(1, nsamp, r0, amp=60.0, seed=2)
    cfg = synth.SearchCfg(zmax=0, numharm=1, whiten_block=64)
    obj = RF.Objective(fil, [synth.Stage(0.0, 1.0, 3, 1)], cfg, dm_idx=0)
    assert obj.grid_max(0.0, r0 - 1.0, 0.0, 1, 1.0, 0.0)[2] == r0
    assert obj.grid_max(0.0, r0 + 1.0, 0.0, 1, 1.0, 0.0)[2] == r0
