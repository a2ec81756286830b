"""GPU parity: every stage of the CUDA path, called through the C ABI,
against the FP64 oracle on the same seeded inputs.

Dedispersion is bit-exact; normalised powers agree within 1e-4 of
max(P, 1); raw candidate sets agree exactly except for points within
0.05 sigma of the threshold or with a neighbour tie within 1e-4."""
import numpy as np
import pytest

from oracle import dedisperse as OD
from oracle import plan as OP
from oracle import response as OR
from oracle import spectrum as OS
from paper_1912_12807_gb300 import synth

from _parity import check_powers, compare_candidates, oracle_plane

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


def _torch_dev(arr):
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr)).cuda()


# ---------------------------------------------------------------- response
def test_response_matches_quadrature(L, ctx):
    rng = np.random.default_rng(0)
    q = np.concatenate([rng.uniform(-120, 120, 150), np.arange(-20, 21) * 0.5, [0.0, 0.25, -0.3]])
    z = np.concatenate([rng.uniform(-200, 200, 150), np.zeros(41), [1e-7, -3e-3, 0.02]])
    z[:10] = np.round(z[:10])
    z[10:20] = rng.uniform(-0.02, 0.02, 10)
    got = L.pss_response(ctx, q, z)
    ref = np.array([OR.rho_quad(a, b) for a, b in zip(q, z)])
    assert np.max(np.abs(got - ref)) < 1e-10


# ---------------------------------------------------------------- dedispersion
def _dd_check(L, ctx, fil, stages, mask=None, layout=0, data=None, sub=None):
    desc = L.FilDesc.of(fil, chan_mask=mask, layout=layout)
    plan = L.Plan(desc, stages)
    op = OP.Plan.for_file(fil, stages)
    x = OD.channel_major(fil.data, fil.nchan, fil.nbits)
    if data is None:
        data = fil.data if layout == 0 else x
    b, e = sub if sub else (0, plan.ndm)
    out = L.pss_dedisperse(ctx, plan, _torch_dev(data), b, e).cpu().numpy()
    off = 0
    for i in range(b, e):
        nv, _ = op.nv_nfft(i)
        ref = OD.dedisperse(x, op.delays[i], op.max_delay, int(op.ds_of[i]), mask)
        np.testing.assert_array_equal(out[off:off + nv], ref, err_msg="DM index %d" % i)
        off += nv
    assert off == out.shape[0]


def test_dedisperse_small_bit_exact(L, ctx, small):
    _dd_check(L, ctx, small.fil, small.stages)


def test_dedisperse_host_input_and_subrange(L, ctx, small):
    fil = small.fil
    desc = L.FilDesc.of(fil)
    plan = L.Plan(desc, small.stages)
    a = L.pss_dedisperse(ctx, plan, fil.data, 17, 40).cpu().numpy()   # host pointer
    b = L.pss_dedisperse(ctx, plan, _torch_dev(fil.data), 17, 40).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    assert L.pss_dedisperse(ctx, plan, fil.data, 5, 5).numel() == 0


@pytest.mark.parametrize("nchan,nsamp,ds", [(48, 20000 + 37, 1), (300, 9000 + 5, 1), (64, 40000 + 11, 4),
                                            (32, 33333, 1024)])
def test_dedisperse_ragged_wide_downsampled(L, ctx, nchan, nsamp, ds):
    fil = synth.make_8bit(nchan, nsamp, 2e-4, 1200.0, 1500.0, [synth.Pulsar(0.05, 30.0, 0.05, 0.8)], seed=nchan)
    stages = [synth.Stage(0.0, 3.0, 13, 1), synth.Stage(39.0, 7.0, 9, ds)]
    _dd_check(L, ctx, fil, stages)


def test_dedisperse_mask_and_channel_major(L, ctx, small):
    mask = np.ones(64, dtype=np.uint8)
    mask[[0, 7, 8, 40, 63]] = 0
    _dd_check(L, ctx, small.fil, small.stages, mask=mask, sub=(30, 70))
    _dd_check(L, ctx, small.fil, small.stages, layout=1, sub=(0, 20))


def test_dedisperse_one_bit(L, ctx):
    fil = synth.make_1bit(96, 1 << 15, 2.5e-4, 1230.0, 1518.0,
                          [synth.Pulsar(0.02, 100.0, 0.05, 0.1)], seed=4)
    stages = synth.stages_from_table([(0.0, 100.0, 5.0, 1), (100.0, 300.0, 10.0, 2), (300.0, 500.0, 25.0, 4)], True)
    _dd_check(L, ctx, fil, stages)


def test_dedisperse_extreme_values(L, ctx):
    # all-255 input: every output is 255 * nchan * ds exactly
    nchan, nsamp = 257, 5000
    fil = synth.make_8bit(nchan, nsamp, 2e-4, 1200.0, 1500.0, [], seed=1)
    fil.data[:] = 255
    stages = [synth.Stage(0.0, 5.0, 9, 1), synth.Stage(45.0, 5.0, 3, 8)]
    desc = L.FilDesc.of(fil)
    plan = L.Plan(desc, stages)
    out = L.pss_dedisperse(ctx, plan, _torch_dev(fil.data), 0, plan.ndm).cpu().numpy()
    op = OP.Plan.for_file(fil, stages)
    off = 0
    for i in range(plan.ndm):
        nv, _ = op.nv_nfft(i)
        assert np.all(out[off:off + nv] == 255 * nchan * int(op.ds_of[i]))
        off += nv


# ---------------------------------------------------------------- spectrum / plane
def _cfg(L, wl, **kw):
    c = L.cfg_of(wl.cfg)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def test_spectrum_and_zmax0_plane(L, ctx, small):
    fil = small.fil
    cfg = _cfg(L, small)
    desc = L.FilDesc.of(fil)
    plan = L.Plan(desc, small.stages)
    op = OP.Plan.for_file(fil, small.stages)
    x = OD.channel_major(fil.data, fil.nchan, 8)
    idx = [0, 1, 49, 50, 51, 100]
    dev = _torch_dev(fil.data)
    for i in idx:
        spec = L.pss_spectrum(ctx, plan, dev, cfg, i, i + 1).cpu().numpy()
        plane = L.pss_power_plane(ctx, plan, dev, cfg, i, i + 1).cpu().numpy()
        _, Ap, ref_plane = oracle_plane(x, op, i, small.cfg)
        check_powers(np.abs(spec) ** 2, np.abs(Ap) ** 2, "spectrum DM %d" % i)
        check_powers(plane, ref_plane[0], "plane DM %d" % i)


@pytest.mark.parametrize("zmax,dz", [(20, 2.0), (50, 2.0), (7, 0.5)])
def test_accel_plane(L, ctx, zmax, dz):
    fil = synth.make_8bit(64, 1 << 14, 2e-4, 1200.0, 1500.0,
                          [synth.Pulsar(0.01, 20.0, 0.05, 0.3, z_direct=9.0)], seed=3)
    stages = [synth.Stage(10.0, 5.0, 4, 1)]
    wl = synth.Workload("t", fil, stages, synth.SearchCfg(zmax=zmax, dz=dz, numharm=4, whiten_block=256))
    cfg = _cfg(L, wl)
    plan = L.Plan(L.FilDesc.of(fil), stages)
    op = OP.Plan.for_file(fil, stages)
    x = OD.channel_major(fil.data, fil.nchan, 8)
    got = L.pss_power_plane(ctx, plan, _torch_dev(fil.data), cfg, 1, 3).cpu().numpy()
    nz = L.n_z(cfg)
    nfft = op.nv_nfft(1)[1]
    for k, i in enumerate((1, 2)):
        _, _, ref = oracle_plane(x, op, i, wl.cfg)
        check_powers(got[k * nz * nfft:(k + 1) * nz * nfft].reshape(nz, nfft), ref, "accel plane DM %d" % i)


@pytest.mark.parametrize("form", ["0", "1"])
def test_accel_plane_both_fft_forms(L, monkeypatch, form):
    # both overlap-save kernels (radix 8-8-8-4 and 16-16-8; an autotuner choice) against the oracle
    monkeypatch.setenv("PSS_PLANE_FORM", form)
    c = L.Context(0)
    fil = synth.make_8bit(64, 1 << 14, 2e-4, 1200.0, 1500.0,
                          [synth.Pulsar(0.01, 20.0, 0.05, 0.3, z_direct=9.0)], seed=3)
    stages = [synth.Stage(10.0, 5.0, 4, 1)]
    for zmax, dz in ((50, 2.0), (7, 0.5)):
        wl = synth.Workload("t", fil, stages, synth.SearchCfg(zmax=zmax, dz=dz, numharm=4, whiten_block=256))
        cfg = _cfg(L, wl)
        plan = L.Plan(L.FilDesc.of(fil), stages)
        op = OP.Plan.for_file(fil, stages)
        x = OD.channel_major(fil.data, fil.nchan, 8)
        got = L.pss_power_plane(c, plan, _torch_dev(fil.data), cfg, 1, 2).cpu().numpy()
        nz, nfft = L.n_z(cfg), op.nv_nfft(1)[1]
        _, _, ref = oracle_plane(x, op, 1, wl.cfg)
        check_powers(got.reshape(nz, nfft), ref, "plane form %s zmax %d" % (form, zmax))
    c.close()


def test_accel_plane_direct_form(L, ctx):
    # a spectrum shorter than the overlap-save segment (1024 bins) takes the direct form
    fil = synth.make_8bit(32, 2000, 2e-4, 1200.0, 1500.0,
                          [synth.Pulsar(0.01, 20.0, 0.05, 0.3, z_direct=5.0)], seed=4)
    stages = [synth.Stage(10.0, 5.0, 3, 1)]
    wl = synth.Workload("t", fil, stages, synth.SearchCfg(zmax=12, dz=2.0, numharm=4, whiten_block=128))
    cfg = _cfg(L, wl)
    plan = L.Plan(L.FilDesc.of(fil), stages)
    op = OP.Plan.for_file(fil, stages)
    x = OD.channel_major(fil.data, fil.nchan, 8)
    nfft = op.nv_nfft(1)[1]
    assert nfft // 2 < 2048
    got = L.pss_power_plane(ctx, plan, _torch_dev(fil.data), cfg, 1, 2).cpu().numpy()
    _, _, ref = oracle_plane(x, op, 1, wl.cfg)
    check_powers(got.reshape(L.n_z(cfg), nfft), ref, "direct-form accel plane")


def test_fused_cluster_spectrum_parity(L, ctx, monkeypatch):
    # nfft = 2^18 at zmax 0 with PSS_FUSED=1 runs the 16-CTA cluster kernel
    # (FFT, whitening and the half-bin plane in distributed shared memory):
    # planes against the oracle, the separate kernels against the same
    # oracle, and the raw detections of the fused path
    fil = synth.make_8bit(32, 1 << 18, 2e-4, 1200.0, 1500.0,
                          [synth.Pulsar(0.0213, 1.0, 0.05, 0.08, phase0=0.3)], seed=11)
    stages = [synth.Stage(0.0, 1.0, 3, 1)]
    wl = synth.Workload("t", fil, stages, synth.SearchCfg(zmax=0, numharm=8))
    cfg = _cfg(L, wl)
    plan = L.Plan(L.FilDesc.of(fil), stages)
    op = OP.Plan.for_file(fil, stages)
    assert op.nv_nfft(0)[1] == 1 << 18
    x = OD.channel_major(fil.data, fil.nchan, 8)
    dev = _torch_dev(fil.data)
    monkeypatch.setenv("PSS_FUSED", "1")
    cf = L.Context(0)
    got = L.pss_power_plane(cf, plan, dev, cfg, 0, 3).cpu().numpy().reshape(3, 1 << 18)
    refs = [oracle_plane(x, op, i, wl.cfg)[2] for i in range(3)]
    for i in range(3):
        check_powers(got[i:i + 1], refs[i], "fused plane DM %d" % i)
    sep = L.pss_power_plane(ctx, plan, dev, cfg, 0, 3).cpu().numpy().reshape(3, 1 << 18)
    for i in range(3):
        check_powers(sep[i:i + 1], refs[i], "separate-kernel plane DM %d" % i)
    raw = L.pss_search_raw(cf, plan, dev, cfg, 0, 3)
    cf.close()
    n = 0
    for i in range(3):
        g, r, e = compare_candidates(raw, refs[i][None, :] if refs[i].ndim == 1 else refs[i], i, 8, 0,
                                     op.t_span(i), wl.cfg.f_lo_hz, wl.cfg.sigma_thr)
        n += r
    assert n > 0


# ---------------------------------------------------------------- candidates
def test_search_raw_small_parity(L, ctx, small):
    fil = small.fil
    cfg = _cfg(L, small)
    plan = L.Plan(L.FilDesc.of(fil), small.stages)
    op = OP.Plan.for_file(fil, small.stages)
    x = OD.channel_major(fil.data, fil.nchan, 8)
    raw = L.pss_search_raw(ctx, plan, _torch_dev(fil.data), cfg, 0, plan.ndm)
    assert np.all(np.diff(raw["dm_idx"]) >= 0)
    tot_ref = 0
    for i in range(0, plan.ndm, 5):
        _, _, pl = oracle_plane(x, op, i, small.cfg)
        g, r, e = compare_candidates(raw, pl, i, small.cfg.numharm, 0, op.t_span(i), small.cfg.f_lo_hz,
                                     small.cfg.sigma_thr)
        tot_ref += r
    assert tot_ref > 100  # the injected pulsar gives many detections near DM 50
    # the sifted list is the sift of the raw list, and finds the pulsar
    cands = L.pss_search_dm_batch(ctx, plan, _torch_dev(fil.data), cfg, 0, plan.ndm)
    again = L.pss_sift(plan, cfg, raw)
    assert cands.tobytes() == again.tobytes()
    best = cands[np.argmax(cands["sigma"])]
    assert abs(best["dm"] - 50.0) <= 1.0
    assert abs(best["f_hz"] - 1 / 0.0333) < 1.0 / (65536 * 2e-4)


def test_pipelined_2d_sift_equals_sift_of_raw(L, ctx):
    # zmax > 0 with 200 trials: the pipelined search links each DM batch's survivors to the
    # earlier ones while the device works (four batches); its list must be the one-pass sift of
    # the raw detections, byte for byte (a low threshold gives many linked groups)
    fil = synth.make_8bit(64, 1 << 15, 2e-4, 1200.0, 1500.0,
                          [synth.Pulsar(0.01, 60.0, 0.05, 0.6, z_direct=6.0), synth.Pulsar(0.0123, 20.0, 0.05, 0.4)],
                          seed=17)
    stages = [synth.Stage(0.0, 0.5, 200, 1)]
    plan = L.Plan(L.FilDesc.of(fil), stages)
    cfg = L.search_cfg(zmax=16, dz=2.0, numharm=8, sigma_thr=3.5, whiten_block=256)
    d = _torch_dev(fil.data)
    raw = L.pss_search_raw(ctx, plan, d, cfg, 0, plan.ndm, cap=1 << 22)
    cands = L.pss_search_dm_batch(ctx, plan, d, cfg, 0, plan.ndm, cap=1 << 18)
    again = L.pss_sift(plan, cfg, raw, cap=1 << 18)
    assert len(cands) > 10 and len(raw) > 10 * len(cands)
    assert cands.tobytes() == again.tobytes()


def test_search_accel_parity(L, ctx):
    fil = synth.make_8bit(64, 1 << 14, 2e-4, 1200.0, 1500.0,
                          [synth.Pulsar(0.01, 20.0, 0.05, 0.6, z_direct=9.0)], seed=3)
    stages = [synth.Stage(10.0, 5.0, 4, 1)]
    wl = synth.Workload("t", fil, stages, synth.SearchCfg(zmax=20, dz=2.0, numharm=4, whiten_block=256))
    cfg = _cfg(L, wl)
    plan = L.Plan(L.FilDesc.of(fil), stages)
    op = OP.Plan.for_file(fil, stages)
    x = OD.channel_major(fil.data, fil.nchan, 8)
    raw = L.pss_search_raw(ctx, plan, _torch_dev(fil.data), cfg, 0, plan.ndm)
    n = 0
    for i in range(plan.ndm):
        _, _, pl = oracle_plane(x, op, i, wl.cfg)
        g, r, e = compare_candidates(raw, pl, i, 4, 10, op.t_span(i), wl.cfg.f_lo_hz, wl.cfg.sigma_thr)
        n += r
    assert n > 0
    assert np.any(raw["j"] != 10)  # detections off the z = 0 row


def test_errors(L, ctx, small):
    fil = small.fil
    plan = L.Plan(L.FilDesc.of(fil), small.stages)
    bad = _cfg(L, small, numharm=3)
    with pytest.raises(L.PssError) as e:
        L.pss_search_raw(ctx, plan, fil.data, bad, 0, 3)
    assert e.value.status == L.PSS_EINVAL
    with pytest.raises(L.PssError):
        L.pss_search_raw(ctx, plan, fil.data, _cfg(L, small), 0, plan.ndm + 1)
    with pytest.raises(L.PssError):
        L.pss_search_raw(ctx, plan, fil.data, _cfg(L, small, whiten_block=100), 0, 3)
    assert L.pss_search_raw(ctx, plan, fil.data, _cfg(L, small), 4, 4).shape[0] == 0
    # capacity: ask for less than needed, get PSS_ECAP and the count
    import ctypes as C
    raw = np.zeros(1, dtype=L.RAW_DTYPE)
    n = C.c_int64()
    st = L.lib().pss_search_raw(ctx.h, plan.h, C.byref(plan.desc.c), C.c_void_p(fil.data.ctypes.data), 0,
                                C.byref(_cfg(L, small)), 45, 55, raw.ctypes.data, 1, C.byref(n), None)
    assert st == L.PSS_ECAP and n.value > 1
