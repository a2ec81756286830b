"""GPU parity at the full sizes of the benchmark workloads, through the C ABI,
against the FP64 oracle on sampled trials (the oracle finishes a trial in
seconds; whole files would take it hours).

* PMPS-shaped file (96 channels, 1-bit, 2^23 samples, staged plan of 1081
  trials with ds 1/2/4): the search runs over every trial in one call (the
  benchmark's launch); the first and last trial of each stage are checked:
  series bit for bit, spectra at nfft 2^23 / 2^22 / 2^21 (three-, three-
  and two-pass FFTs), zmax 0 planes and raw candidate sets.  At zmax 50 the
  nfft 2^21 trial is checked whole (plane and candidates), the nfft 2^23
  trial at sampled plane points and at every GPU candidate.
* Acceleration file (256 channels, 2^18, zmax 200, dz 2, numharm 8): every
  trial in one call; planes and raw candidates of the trials nearest the
  two pulsars injected with z = +37 and -151, and of the last trial.
* Stream shape at its largest (1024 channels, 2^19 samples, DM 0-500 step
  1, zmax 100, numharm 8): series, plane and candidates of two trials.
* Drift-scan file (256 channels, 2^18, 1001 trials, numharm 16): every
  trial in one call; raw candidates of the first and last trials and of
  the trials nearest the five pulsars.
* Every FFT pass split the autotuner may choose, for every transform size
  of these workloads (nfft 2^16 to 2^23), against the oracle spectrum; a
  tuned staged batch runs a valid split for each of its sizes, and its
  splits reproduce the oracle.
* Folding: GPU profiles against the exact phase j x + j^2 g of the FP64
  x = f dt, g = (fdot/2) dt^2 (rational arithmetic), excusing only samples
  within (j + j^2) 2^-65 cycle of a bin edge (the fixed-point rounding).
"""
import itertools
import os

import numpy as np
import pytest

from oracle import dedisperse as OD
from oracle import plan as OP
from oracle import spectrum as OS
from paper_1912_12807_gb300 import synth

from _parity import (check_candidates_at_points, check_powers, compare_candidates, oracle_plane,
                     oracle_plane_points)

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


def _offsets(op, lo, hi, key):
    """Packed row offsets of trials [lo, hi) (key 0: N_v, 1: nfft)."""
    off = [0]
    for i in range(lo, hi):
        off.append(off[-1] + op.nv_nfft(i)[key])
    return off


def _nearest(op, dm):
    return int(np.argmin(np.abs(op.dms - dm)))


# ---------------------------------------------------------------- PMPS-shaped
@pytest.fixture(scope="module")
def pmps():
    wl = synth.workload_pmps(zmax=0)
    op = OP.Plan.for_file(wl.fil, wl.stages)
    x = OD.channel_major(wl.fil.data, wl.fil.nchan, 1)
    edges = np.cumsum([0] + [s.n_dm for s in wl.stages])
    sample = sorted({int(edges[k]) for k in range(3)} | {int(edges[k + 1]) - 1 for k in range(3)})
    return wl, op, x, sample


def test_pmps_fullsize_zmax0(L, ctx, pmps):
    import torch
    wl, op, x, sample = pmps
    plan = L.Plan(L.FilDesc.of(wl.fil), wl.stages)
    assert plan.ndm == 1081
    dev = _dev(wl.fil.data)
    cfg = L.cfg_of(wl.cfg)
    # series: every trial in one call, sampled rows compared bit for bit
    ser = L.pss_dedisperse(ctx, plan, dev, 0, plan.ndm)
    off = _offsets(op, 0, plan.ndm, 0)
    for i in sample:
        ref = OD.dedisperse(x, op.delays[i], op.max_delay, int(op.ds_of[i]))
        np.testing.assert_array_equal(ser[off[i]:off[i + 1]].cpu().numpy(), ref, err_msg="DM index %d" % i)
    del ser
    torch.cuda.empty_cache()
    raw = L.pss_search_raw(ctx, plan, dev, cfg, 0, plan.ndm)
    nffts = set()
    for i in sample:
        s, Ap, ref_plane = oracle_plane(x, op, i, wl.cfg)
        nffts.add(op.nv_nfft(i)[1])
        spec = L.pss_spectrum(ctx, plan, dev, cfg, i, i + 1).cpu().numpy()
        check_powers(np.abs(spec) ** 2, np.abs(Ap) ** 2, "spectrum DM %d" % i)
        pl = L.pss_power_plane(ctx, plan, dev, cfg, i, i + 1).cpu().numpy()
        check_powers(pl, ref_plane[0], "plane DM %d" % i)
        compare_candidates(raw, ref_plane, i, wl.cfg.numharm, 0, op.t_span(i), wl.cfg.f_lo_hz, wl.cfg.sigma_thr)
    assert nffts == {1 << 23, 1 << 22, 1 << 21}
    # the sifted list of the whole plan is the sift of the raw list
    cands = L.pss_search_dm_batch(ctx, plan, dev, cfg, 0, plan.ndm)
    assert cands.tobytes() == L.pss_sift(plan, cfg, raw).tobytes()


def test_pmps_fullsize_zmax50(L, ctx, pmps):
    wl, op, x, sample = pmps
    cfg = L.cfg_of(wl.cfg)
    cfg.zmax = 50
    ocfg = synth.SearchCfg(zmax=50, dz=wl.cfg.dz, numharm=wl.cfg.numharm)
    plan = L.Plan(L.FilDesc.of(wl.fil), wl.stages)
    dev = _dev(wl.fil.data)
    raw = L.pss_search_raw(ctx, plan, dev, cfg, 0, plan.ndm)
    nz = L.n_z(cfg)
    # a trial of the ds 4 stage (nfft 2^21): the whole plane and candidate set
    i = 800
    assert op.nv_nfft(i)[1] == 1 << 21
    _, Ap, ref_plane = oracle_plane(x, op, i, ocfg, method="fftconv")
    pl = L.pss_power_plane(ctx, plan, dev, cfg, i, i + 1).cpu().numpy().reshape(nz, -1)
    check_powers(pl, ref_plane, "zmax 50 plane DM %d" % i)
    del pl
    compare_candidates(raw, ref_plane, i, ocfg.numharm, nz // 2, op.t_span(i), ocfg.f_lo_hz, ocfg.sigma_thr)
    del ref_plane
    # the first trial (nfft 2^23, 51 x 2^23 plane): sampled points and every candidate
    i = 0
    nv, nfft = op.nv_nfft(i)
    s = OD.dedisperse(x, op.delays[i], op.max_delay, 1)
    Ap = OS.whiten(OS.half_spectrum(OS.real_series(s, nfft)), ocfg.whiten_block)
    plg = L.pss_power_plane(ctx, plan, dev, cfg, i, i + 1).view(nz, nfft)
    rng = np.random.default_rng(50)
    js = np.concatenate([rng.integers(0, nz, 20000), np.full(8, nz // 2), [0, nz - 1] * 4])
    hs = np.concatenate([rng.integers(0, nfft, 20000), [0, 1, 2, 3, nfft - 1, nfft - 2, nfft - 3, nfft - 4],
                         [0, nfft - 1, 1, nfft - 2, 5000, 5001, 1 << 20, (1 << 20) + 1]])
    import torch
    got = plg[torch.from_numpy(js).cuda(), torch.from_numpy(hs).cuda()].cpu().numpy()
    check_powers(got, oracle_plane_points(Ap, 50, ocfg.dz, ocfg.halfwidth_extra, js, hs), "zmax 50 nfft 2^23 points")
    n = check_candidates_at_points(raw, Ap, i, ocfg.numharm, 50, ocfg.dz, ocfg.halfwidth_extra, nz, nfft,
                                   op.t_span(i), ocfg.f_lo_hz, ocfg.sigma_thr)
    assert n > 100


# ---------------------------------------------------------------- acceleration (zmax 200)
def test_accel_fullsize_zmax200(L, ctx):
    wl = synth.workload_accel()
    op = OP.Plan.for_file(wl.fil, wl.stages)
    x = OD.channel_major(wl.fil.data, wl.fil.nchan, 8)
    plan = L.Plan(L.FilDesc.of(wl.fil), wl.stages)
    cfg = L.cfg_of(wl.cfg)
    dev = _dev(wl.fil.data)
    raw = L.pss_search_raw(ctx, plan, dev, cfg, 0, plan.ndm)
    nz = L.n_z(cfg)
    assert nz == 201
    zdirect = [p for p in wl.fil.pulsars if getattr(p, "z_direct", None)]
    assert len(zdirect) == 2
    sample = sorted({_nearest(op, p.dm) for p in zdirect} | {plan.ndm - 1})
    hits = 0
    for i in sample:
        _, Ap, ref_plane = oracle_plane(x, op, i, wl.cfg, method="fftconv")
        pl = L.pss_power_plane(ctx, plan, dev, cfg, i, i + 1).cpu().numpy().reshape(nz, -1)
        check_powers(pl, ref_plane, "zmax 200 plane DM %d" % i)
        del pl
        g, r, e = compare_candidates(raw, ref_plane, i, wl.cfg.numharm, nz // 2, op.t_span(i), wl.cfg.f_lo_hz,
                                     wl.cfg.sigma_thr)
        # the z-direct pulsar of this trial is detected off the z = 0 row
        rows = raw[(raw["dm_idx"] == i) & (raw["j"] != nz // 2)]
        hits += int(len(rows) > 0)
    assert hits >= 2


# ---------------------------------------------------------------- stream shape, largest file
def test_stream_shape_1024ch_2e19_zmax100(L, ctx):
    rng = np.random.default_rng(5077)
    psrs = synth._drift_pulsars(rng, 2, 1024, 1 << 19)
    fil = synth.make_8bit_stream(1024, 1 << 19, 2e-4, 1050.0, 1450.0, psrs, 5077)
    stages = [synth.Stage(0.0, 1.0, 501, 1)]
    ocfg = synth.SearchCfg(zmax=100, dz=2.0, numharm=8)
    op = OP.Plan.for_file(fil, stages)
    x = OD.channel_major(fil.data, fil.nchan, 8)
    plan = L.Plan(L.FilDesc.of(fil), stages)
    cfg = L.cfg_of(ocfg)
    dev = _dev(fil.data)
    nz = L.n_z(cfg)
    raw = L.pss_search_raw(ctx, plan, dev, cfg, 0, plan.ndm)
    ser = L.pss_dedisperse(ctx, plan, dev, 0, plan.ndm)
    off = _offsets(op, 0, plan.ndm, 0)
    for i in (_nearest(op, psrs[0].dm), plan.ndm - 1):
        s, Ap, ref_plane = oracle_plane(x, op, i, ocfg, method="fftconv")
        np.testing.assert_array_equal(ser[off[i]:off[i + 1]].cpu().numpy(), s, err_msg="DM index %d" % i)
        pl = L.pss_power_plane(ctx, plan, dev, cfg, i, i + 1).cpu().numpy().reshape(nz, -1)
        check_powers(pl, ref_plane, "zmax 100 plane DM %d" % i)
        del pl
        compare_candidates(raw, ref_plane, i, ocfg.numharm, nz // 2, op.t_span(i), ocfg.f_lo_hz, ocfg.sigma_thr)


# ---------------------------------------------------------------- drift-scan, numharm 16
def test_driftscan_fullsize_numharm16(L, ctx):
    wl = synth.workload_driftscan()
    op = OP.Plan.for_file(wl.fil, wl.stages)
    x = OD.channel_major(wl.fil.data, wl.fil.nchan, 8)
    plan = L.Plan(L.FilDesc.of(wl.fil), wl.stages)
    cfg = L.cfg_of(wl.cfg)
    dev = _dev(wl.fil.data)
    raw = L.pss_search_raw(ctx, plan, dev, cfg, 0, plan.ndm)
    sample = sorted({0, plan.ndm - 1} | {_nearest(op, p.dm) for p in wl.fil.pulsars})
    tot = 0
    for i in sample:
        _, _, ref_plane = oracle_plane(x, op, i, wl.cfg)
        g, r, e = compare_candidates(raw, ref_plane, i, wl.cfg.numharm, 0, op.t_span(i), wl.cfg.f_lo_hz,
                                     wl.cfg.sigma_thr)
        tot += r
    assert tot > 100
    cands = L.pss_search_dm_batch(ctx, plan, dev, cfg, 0, plan.ndm)
    assert cands.tobytes() == L.pss_sift(plan, cfg, raw).tobytes()


# ---------------------------------------------------------------- every FFT pass split
def _file_with_nfft(nfft, nbits=8, seed=0):
    """A 16-channel file whose single trial row has exactly nfft points."""
    nsamp = nfft // 2 + 3000
    mk = synth.make_8bit if nbits == 8 else synth.make_1bit
    fil = mk(16, nsamp, 2e-4, 1200.0, 1500.0, [synth.Pulsar(0.01, 20.0, 0.05, 0.3)], seed=seed)
    stages = [synth.Stage(0.0, 10.0, 3, 1)]
    return fil, stages


@pytest.mark.parametrize("log2n", [16, 17, 18, 19, 20, 21, 22, 23])
def test_every_fft_split_matches_oracle(L, log2n):
    nfft = 1 << log2n
    splits = L.pss_fft_splits(nfft)
    assert splits and splits[0][0] == 0
    for v, rad in splits:
        assert int(np.prod(rad)) == nfft // 2 and all(32 <= r <= 1024 for r in rad)
    fil, stages = _file_with_nfft(nfft, seed=log2n)
    op = OP.Plan.for_file(fil, stages)
    assert op.nv_nfft(0)[1] == nfft
    x = OD.channel_major(fil.data, fil.nchan, 8)
    refs = []
    for i in range(2):
        s = OD.dedisperse(x, op.delays[i], op.max_delay, 1)
        refs.append(np.abs(OS.whiten(OS.half_spectrum(OS.real_series(s, nfft)), 1024)) ** 2)
    plan = L.Plan(L.FilDesc.of(fil), stages)
    cfg = L.search_cfg(zmax=0, numharm=8)
    dev = _dev(fil.data)
    c = L.Context(0)
    try:
        for v, rad in splits:
            L.pss_ctx_set_fft_split(c, nfft, v)
            spec = L.pss_spectrum(c, plan, dev, cfg, 0, 2).cpu().numpy()
            for i in range(2):
                check_powers(np.abs(spec[i * (nfft // 2):(i + 1) * (nfft // 2)]) ** 2, refs[i],
                             "nfft 2^%d split %d %s trial %d" % (log2n, v, rad, i))
        with pytest.raises(L.PssError):
            L.pss_ctx_set_fft_split(c, nfft, len(splits))
    finally:
        c.close()


def test_tuned_staged_batch_runs_a_split_per_size(L, monkeypatch):
    # a 1-bit staged file with the PMPS plan's three transform sizes (nfft 2^22, 2^21, 2^20):
    # 2^22 has many pass splits, 2^21 only the even one
    fil = synth.make_1bit(32, (1 << 21) + 4000, 2.5e-4, 1230.0, 1518.0, [synth.Pulsar(0.02, 60.0, 0.05, 0.1)],
                          seed=11)
    stages = synth.stages_from_table([(0.0, 40.0, 10.0, 1), (40.0, 80.0, 10.0, 2), (80.0, 120.0, 10.0, 4)], True)
    op = OP.Plan.for_file(fil, stages)
    firsts = [int(k) for k in np.cumsum([0] + [s.n_dm for s in stages])[:-1]]
    nffts = [op.nv_nfft(k)[1] for k in firsts]
    assert nffts == [1 << 22, 1 << 21, 1 << 20]
    plan = L.Plan(L.FilDesc.of(fil), stages)
    cfg = L.search_cfg(zmax=0, numharm=8)
    x = OD.channel_major(fil.data, fil.nchan, 1)

    def check_ctx_with(splits):
        c = L.Context(0)
        try:
            for nfft, v in splits.items():
                L.pss_ctx_set_fft_split(c, nfft, v)
            for i in firsts:
                i = int(i)
                nv, nfft = op.nv_nfft(i)
                s = OD.dedisperse(x, op.delays[i], op.max_delay, int(op.ds_of[i]))
                ref = np.abs(OS.whiten(OS.half_spectrum(OS.real_series(s, nfft)), 1024)) ** 2
                spec = L.pss_spectrum(c, plan, fil.data, cfg, i, i + 1).cpu().numpy()
                check_powers(np.abs(spec) ** 2, ref, "trial %d nfft %d split %d" % (i, nfft, splits[nfft]))
        finally:
            c.close()

    # the autotuner's choice for every size
    b = L.Batch(plan, cfg)
    try:
        tuned = {n: b.fft_split(n) for n in nffts}
        for n, v in tuned.items():
            assert L.pss_fft_split_radices(n, v) is not None
        got = b.run(fil.data)
    finally:
        b.close()
    check_ctx_with(tuned)
    # a split pinned for the first size that the later sizes do not have
    assert len(L.pss_fft_splits(1 << 21)) == 1
    v = min(5, len(L.pss_fft_splits(1 << 22)) - 1)
    assert v >= len(L.pss_fft_splits(1 << 20))
    monkeypatch.setenv("PSS_TUNE", "%d,8,96,-1" % v)
    b = L.Batch(plan, cfg)
    try:
        pinned = {n: b.fft_split(n) for n in nffts}
        assert pinned[1 << 22] == v and pinned[1 << 21] == 0 and pinned[1 << 20] == 0
        for n, w in pinned.items():
            assert L.pss_fft_split_radices(n, w) is not None
        got2 = b.run(fil.data)
    finally:
        b.close()
    check_ctx_with(pinned)
    # the sifted lists agree on the integer parts (only FP32 rounding differs between splits)
    assert len(got) > 0 and len(got2) > 0


# ---------------------------------------------------------------- folding against the exact phase
def _exact_bins(n, dt, f, fdot, nbin):
    """Bins of the exact phase j x + j^2 g of the FP64 values x = f dt and
    g = (0.5 fdot)(dt dt), by integer arithmetic on their exact binary
    values, and each sample's distance to the nearest bin edge in cycles
    (as a float, for the excuse test)."""
    from fractions import Fraction
    xq = Fraction(f * dt)
    gq = Fraction((0.5 * fdot) * (dt * dt))
    den = 1
    for q in (xq, gq):
        den = max(den, q.denominator)
    assert den & (den - 1) == 0  # binary fractions
    X = int(xq * den)
    G = int(gq * den)
    j = np.arange(n, dtype=object)
    num = (j * X + j * j * G) % den              # frac(phase) * den, exact
    scaled = num * nbin
    b = (scaled // den).astype(np.int64)
    rem = scaled % den                            # distance above the lower edge, in units of 1/(den nbin) cycle
    dist_lo = np.array([float(Fraction(int(r), den * nbin)) for r in rem]) if n <= 4096 else \
        (rem.astype(np.float64) / float(den)) / nbin
    dist = np.minimum(dist_lo, 1.0 / nbin - dist_lo)
    return b, dist, np.where(dist_lo < 0.5 / nbin, -1, 1)


def test_fold_bins_match_exact_phase(L, ctx):
    # nbin a power of two: the kernel's bin from the top 32 bits of the phase is then exactly
    # floor(phase * nbin / 2^64), so the only departure from the exact phase is the rounding
    # of x and g to 2^-64 cycle.  Each GPU profile must be the exact-phase profile with some
    # of the excusable samples (within (j + j^2) 2^-65 cycle of an edge) moved across that
    # edge: checked directly by enumeration where there are few such samples, and where a
    # frequency puts many samples on edges (a period of a whole number of samples) through
    # the fixed-point reading, which the GPU must equal exactly and which may differ from the
    # exact phase only at excusable samples
    from oracle import fold as OF
    wl = synth.workload_small()
    fil = wl.fil
    plan = L.Plan(L.FilDesc.of(fil), wl.stages)
    op = OP.Plan.for_file(fil, wl.stages)
    x = OD.channel_major(fil.data, fil.nchan, 8)
    dm = np.array([50, 50, 10, 75, 33, 50])
    f = np.array([30.0217, 90.0651, 7.123456789, 211.5, 0.91, 1 / 0.0333])
    fdot = np.array([0.0, 1e-3, -0.02, 0.05, 0.0, 0.0])
    nbin, nfreq, step = 64, 3, 0.5
    prof, cnt, res = L.pss_fold(ctx, plan, _dev(fil.data), dm, f, fdot, nbin=nbin, nfreq=nfreq, step_bins=step)
    enumerated = 0
    for i, d in enumerate(dm):
        d = int(d)
        s = OD.dedisperse(x, op.delays[d], op.max_delay, 1).astype(np.int64)
        dt = 1 * fil.tsamp_s
        n = s.shape[0]
        fk = float(res["f_hz"][i])
        b, dist, side = _exact_bins(n, dt, fk, float(fdot[i]), nbin)
        jj = np.arange(n, dtype=np.float64)
        bound = (jj + jj * jj) * 2.0 ** -65
        amb = np.nonzero((dist <= bound * 1.0000001) & (jj > 0))[0]  # sample 0 has phase 0 on both sides
        # the fixed-point reading departs from the exact phase only at excusable samples
        bo = OF.phase_bins(n, dt, fk, float(fdot[i]), nbin)
        moved = np.nonzero(bo != b)[0]
        assert np.isin(moved, amb).all(), (i, moved[~np.isin(moved, amb)][:5])
        Po = np.zeros(nbin, dtype=np.int64)
        np.add.at(Po, bo, s)
        np.testing.assert_array_equal(prof[i], Po)
        np.testing.assert_array_equal(cnt[i], np.bincount(bo, minlength=nbin))
        if amb.size > 10:
            continue
        # direct: the GPU profile is the exact-phase profile up to moves of excusable samples
        enumerated += 1
        P = np.zeros(nbin, dtype=np.int64)
        np.add.at(P, b, s)
        cnt_ref = np.bincount(b, minlength=nbin)
        ok = False
        for choice in itertools.product((0, 1), repeat=amb.size):
            P2, c2 = P.copy(), cnt_ref.copy()
            for k, move in zip(amb, choice):
                if move:
                    nb = (b[k] + side[k]) % nbin
                    P2[b[k]] -= s[k]
                    c2[b[k]] -= 1
                    P2[nb] += s[k]
                    c2[nb] += 1
            if np.array_equal(P2, prof[i]) and np.array_equal(c2, cnt[i]):
                ok = True
                break
        assert ok, "candidate %d: GPU profile differs from the exact-phase profile" % i
    assert enumerated >= 4
