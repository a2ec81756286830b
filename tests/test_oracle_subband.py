"""Pins for the two-stage (subband) dedispersion oracle (oracle/subband.py)."""
import numpy as np
import pytest

from oracle import dedisperse as DD
from oracle import plan as P
from oracle import subband as SB
from paper_1912_12807_gb300 import synth

STAGES = [synth.Stage(0.0, 1.0, 13, 1), synth.Stage(13.0, 2.0, 9, 2)]


def _file(nchan=32, nsamp=3000, seed=5):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 256, size=(nchan, nsamp)).astype(np.uint8)


def _plans(nchan, nsamp, ts, fch0, foff, stages, sub):
    return (P.Plan(nchan, nsamp, ts, fch0, foff, stages),
            P.Plan(nchan, nsamp, ts, fch0, foff, stages, subband=sub))


@pytest.mark.parametrize("foff", [3.0, -3.0])
def test_one_channel_subbands_are_exact(foff):
    # S = 1: e_c = 0 and D_b(i) = d_c(i), the textbook shift-and-sum.
    x = _file()
    mask = np.ones(32, bool)
    mask[[3, 17]] = False
    ex, sb = _plans(32, 3000, 5e-4, 1200.0, foff, STAGES, (32, 4))
    assert sb.max_delay == ex.max_delay
    assert np.array_equal(sb.sub.D, ex.delays)
    for i in range(len(ex.dms)):
        ds = int(ex.ds_of[i])
        ref = DD.dedisperse(x, ex.delays[i], ex.max_delay, ds, mask)
        got = SB.dedisperse_subband(x, sb.sub, i, sb.max_delay, ds, mask)
        assert np.array_equal(ref, got), i


def test_one_subband_groups_of_one_are_exact():
    # nsub = 1, group = 1: f_b = f_ref, D_0 = 0 and e_c at the trial's own DM.
    x = _file()
    ex, sb = _plans(32, 3000, 5e-4, 1200.0, 3.0, STAGES, (1, 1))
    assert np.array_equal(sb.sub.e, ex.delays)
    assert not sb.sub.D.any()
    for i in range(len(ex.dms)):
        ds = int(ex.ds_of[i])
        assert np.array_equal(DD.dedisperse(x, ex.delays[i], ex.max_delay, ds),
                              SB.dedisperse_subband(x, sb.sub, i, sb.max_delay, ds))


def test_single_sum_brute_force():
    # s[t] = sum_c x[c][t + e_c(g) + D_b(c)(i)] by a pure-Python loop, then
    # the boxcar: the two stages only regroup this sum.
    x = _file(16, 900, 7)
    mask = [c % 5 != 2 for c in range(16)]
    _, sb = _plans(16, 900, 1e-3, 1100.0, 6.0, [synth.Stage(5.0, 3.0, 7, 1), synth.Stage(26.0, 4.0, 5, 2)],
                   (4, 3))
    L = 900 - sb.max_delay
    for i in range(len(sb.dms)):
        comb = sb.sub.combined_delays(i)
        s = [sum(int(x[c][t + int(comb[c])]) for c in range(16) if mask[c]) for t in range(L)]
        ds = int(sb.ds_of[i])
        ref = [sum(s[j * ds:(j + 1) * ds]) for j in range(L // ds)]
        assert SB.dedisperse_subband(x, sb.sub, i, sb.max_delay, ds, mask).tolist() == ref


def test_combined_delay_above_the_exact_maximum_bounds_the_valid_length():
    # With groups of one, e_c + D_b rounds twice: 64 channels in 8 subbands,
    # DM 0-11.4 in steps of 0.6 reach a combined delay of 59 samples where the
    # exact table's largest delay is 58.  The valid length then follows from
    # 59, and every trial still reads inside the file.
    fch0, foff = synth.band(1200.0, 1500.0, 64)
    nsamp = 400
    ex, sb = _plans(64, nsamp, 2e-4, fch0, foff, [synth.Stage(0.0, 0.6, 20, 1)], (8, 1))
    assert ex.max_delay == 58 and sb.sub.max_comb == 59 and sb.max_delay == 59
    assert sb.lengths[0] == (nsamp - 59, 512)
    x = _file(64, nsamp, 9)
    for i in range(len(sb.dms)):
        comb = sb.sub.combined_delays(i)
        assert comb.max() <= sb.max_delay
        want = sum(x[c, int(comb[c]):int(comb[c]) + nsamp - 59].astype(np.int64) for c in range(64))
        assert np.array_equal(SB.dedisperse_subband(x, sb.sub, i, sb.max_delay, 1), want), i


def test_groups_and_nominal_dms():
    _, sb = _plans(32, 3000, 5e-4, 1200.0, 3.0, STAGES, (8, 4))
    g = sb.sub
    # stage 0 (13 trials): groups of 4, 4, 4, 1; stage 1 (9 trials): 4, 4, 1
    assert g.grp_n.tolist() == [4, 4, 4, 1, 4, 4, 1]
    assert g.grp_first.tolist() == [0, 4, 8, 12, 13, 17, 21]
    # the middle (lower middle) trial's DM
    assert g.grp_dm.tolist() == [1.0, 5.0, 9.0, 12.0, 15.0, 23.0, 29.0]
    assert g.grp_of.tolist() == [0] * 4 + [1] * 4 + [2] * 4 + [3] + [4] * 4 + [5] * 4 + [6]
    # f_b = the highest centre frequency of the subband (channels 4b..4b+3)
    assert g.fsub.tolist() == [1200.0 + 3.0 * (4 * b + 3) for b in range(8)]


def test_delay_error_within_the_smearing_bound():
    # |e_c(g) + D_b(i) - d_c(i)| <= |K (DM_i - DM_g) (1/f_c^2 - 1/f_b^2)| / tsamp + 3/2:
    # the three delays are roundings of terms that add up to the exact one
    # except for the DM offset of the within-subband part.
    nchan, ts = 256, 2e-4
    fch0, foff = 1050.78125, 1.5625
    ex, sb = _plans(nchan, 1 << 18, ts, fch0, foff, [synth.Stage(0.0, 0.5, 1001, 1)], (16, 16))
    f = P.channel_freqs(nchan, fch0, foff)
    fb = np.repeat(sb.sub.fsub, 16)
    dmg = sb.sub.grp_dm[sb.sub.grp_of]
    bound = np.abs(P.K_DM * (ex.dms - dmg)[:, None] * (1 / f**2 - 1 / fb**2)[None, :]) / ts + 1.5
    comb = sb.sub.e[sb.sub.grp_of] + np.repeat(sb.sub.D, 16, axis=1)
    err = np.abs(comb - ex.delays)
    assert (err <= bound).all()
    # and the bound is tight enough to matter: trials at their group's nominal DM are exact to 1.5
    at_nom = ex.dms == dmg
    assert (err[at_nom] <= 1).all()
    assert sb.max_delay >= ex.max_delay


def test_injected_pulse_recovered_nearly_at_full_height():
    # A dispersed pulse dedispersed by the two stages peaks at the trial
    # nearest its DM, at no less than 80 % of the exact scheme's peak.
    nchan, N, ts = 64, 1 << 14, 2e-4
    fil = synth.make_8bit(nchan, N, ts, 1200.0, 1500.0,
                          [synth.Pulsar(1.0, 60.0, 0.0006, 40.0, phase0=0.5)], seed=9)
    stages = [synth.Stage(40.0, 1.0, 41, 1)]
    ex = P.Plan.for_file(fil, stages)
    sb = P.Plan.for_file(fil, stages, (8, 8))
    x = DD.channel_major(fil.data, nchan, 8)
    pk_ex = [DD.dedisperse(x, ex.delays[i], ex.max_delay, 1).max() for i in range(len(ex.dms))]
    pk_sb = [SB.dedisperse_subband(x, sb.sub, i, sb.max_delay, 1).max() for i in range(len(sb.dms))]
    base = float(np.median(pk_ex))
    assert abs(sb.dms[int(np.argmax(pk_sb))] - 60.0) <= 1.0
    assert max(pk_sb) - base >= 0.8 * (max(pk_ex) - base)


def test_bad_arguments():
    with pytest.raises(ValueError):
        P.Plan(30, 3000, 5e-4, 1200.0, 3.0, STAGES, subband=(8, 4))   # 8 does not divide 30
    with pytest.raises(ValueError):
        P.Plan(32, 3000, 5e-4, 1200.0, 3.0, STAGES, subband=(8, 0))
