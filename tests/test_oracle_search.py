"""End-to-end oracle check on the small 64-channel workload: the injected
pulsar (P = 33.3 ms, DM 50) is the most significant sifted candidate, found
at its DM and at its fundamental frequency within one Fourier bin."""
from oracle import search
from paper_1912_12807_gb300 import synth


def test_small_workload_finds_injected_pulsar():
    wl = synth.workload_small()
    raw, sifted = search.search(wl.fil, wl.stages, wl.cfg, dm_indices=range(44, 57))
    best = max(sifted, key=lambda c: c["sigma"])
    T = 65536 * 2e-4
    assert abs(best["dm"] - 50.0) <= 1.0
    assert abs(best["f_hz"] - 1.0 / 0.0333) <= 1.0 / T
    assert best["sigma"] > 20
    # every raw candidate passes its stage threshold and lies above f_lo
    for lst in raw.values():
        for c in lst:
            assert c["sigma"] >= 6.0 - 1e-9
            assert c["f_hz"] >= wl.cfg.f_lo_hz - 1e-12


def test_downsampled_stage_reports_the_same_frequency():
    # A stage that sums pairs of samples (ds = 2) transforms half as many
    # points over the same time span: the pulsar's frequency in Hz, and so its
    # fundamental's bin r = f T with T = nfft * ds * tsamp, are unchanged.
    wl = synth.workload_small()
    stages = [synth.Stage(44.0, 1.0, 13, 2)]
    raw, sifted = search.search(wl.fil, stages, wl.cfg)
    best = max(sifted, key=lambda c: c["sigma"])
    T = 32768 * 2 * 2e-4
    assert abs(best["dm"] - 50.0) <= 1.0
    assert abs(best["f_hz"] - 1.0 / 0.0333) <= 1.0 / T
