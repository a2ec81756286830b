"""Host-side checks of libpss that need no GPU: the shared library loads,
exports every symbol include/pss.h declares, has the struct layout the
binding assumes, and its host-only calls (plan, statistics, sift) agree
with the oracle."""
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import plan as OP
from oracle import sift as OS
from oracle import stats as OST
from paper_1912_12807_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1912_12807_gb300 import build, pss
    if not os.path.exists(pss.LIB_PATH):
        build.build()
    return pss


def _declared():
    txt = open(os.path.join(ROOT, "include", "pss.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pss_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    lib = L.lib()
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(L.EXPORTS) == names


def test_struct_layout_matches_binding(L):
    import ctypes as C
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "pss.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %d %zu %zu\n", sizeof(pss_fil_desc), sizeof(pss_dd_stage), sizeof(pss_search_cfg),
         sizeof(pss_raw_cand), sizeof(pss_cand), offsetof(pss_cand, power), offsetof(pss_fil_desc, chan_mask),
         PSS_NPROF_STAGES, sizeof(pss_peaks), offsetof(pss_peaks, lds_bytes_per_s));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(x) for x in subprocess.check_output([exe]).split()]
    want = [C.sizeof(L.pss_fil_desc), C.sizeof(L.pss_dd_stage), C.sizeof(L.pss_search_cfg),
            L.RAW_DTYPE.itemsize, L.CAND_DTYPE.itemsize, L.CAND_DTYPE.fields["power"][1],
            L.pss_fil_desc.chan_mask.offset, len(L.PROFILE_STAGES), C.sizeof(L.pss_peaks),
            L.pss_peaks.lds_bytes_per_s.offset]
    assert got == want


def test_version_and_no_device_error(L):
    assert "sm_103a" in L.pss_version()
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(L.PssError) as e:
        L.Context(0)
    assert e.value.status in (L.PSS_ECUDA, L.PSS_EINVAL)
    desc = L.FilDesc(64, 1 << 14, 2e-4, 1202.34375, 4.6875)
    plan = L.Plan(desc, [synth.Stage(0.0, 1.0, 8, 1)])
    with pytest.raises(L.PssError) as e:
        L.Batch(plan, L.search_cfg())
    assert e.value.status in (L.PSS_ECUDA, L.PSS_EINVAL)
    with pytest.raises(L.PssError) as e:
        L.Server(1 << 30, 2)
    assert e.value.status in (L.PSS_ECUDA, L.PSS_EINVAL)


def test_search_footprint_counts_the_boxcar_table(L, monkeypatch):
    # a row of ds 8 dedisperses from a uint16 table of C x ds x ceil(N/ds) (rows of 8)
    nchan, nsamp, ds = 64, 100000, 8
    desc = L.FilDesc(nchan, nsamp, 2e-4, *synth.band(1200.0, 1500.0, nchan))
    plan = L.Plan(desc, [synth.Stage(0.0, 1.0, 40, ds)])
    cfg = L.search_cfg(zmax=0, numharm=8)
    monkeypatch.delenv("PSS_DEDISP_BX_MIN", raising=False)
    on = L.pss_search_footprint(plan, cfg)
    monkeypatch.setenv("PSS_DEDISP_BX_MIN", "0")
    off = L.pss_search_footprint(plan, cfg)
    table = nchan * ds * (((nsamp + ds - 1) // ds + 7) // 8 * 8) * 2
    assert on - off == table + table // 8 + 256


def test_search_footprint_is_host_arithmetic(L):
    """The admission estimate: at least the buffers one batch of trials
    needs (file, series, three spectra, plane), within 15 % + 64 MiB of
    them, growing with zmax; the checks pss_batch_create makes."""
    nchan, nsamp, nfft = 256, 1 << 18, 1 << 18
    desc = L.FilDesc(nchan, nsamp, 2e-4, *synth.band(1050.0, 1450.0, nchan))
    plan = L.Plan(desc, [synth.Stage(0.0, 0.5, 1001, 1)])
    got0 = L.pss_search_footprint(plan, L.search_cfg(zmax=0, numharm=16))
    B = 1024  # trials per batch: 6 GiB / (20 + 4 nz) bytes per point, at most 1024
    base = nchan * nsamp + B * nfft * 4 + 3 * B * (nfft // 2) * 8
    assert base + B * nfft * 4 <= got0 <= 1.15 * (base + B * nfft * 4) + (64 << 20)
    got50 = L.pss_search_footprint(plan, L.search_cfg(zmax=50, dz=2.0, numharm=16))
    B50 = (6 << 30) // (nfft * (20 + 4 * 51))
    assert got50 >= nchan * nsamp + B50 * 51 * nfft * 4
    with pytest.raises(L.PssError) as e:
        L.pss_search_footprint(plan, L.search_cfg(numharm=3))
    assert e.value.status == L.PSS_EINVAL


@pytest.mark.parametrize("wl", ["small", "drift", "pmps"])
def test_plan_delay_table_bit_exact(L, wl):
    shapes = {
        "small": (64, 1 << 16, 2e-4, 1200.0, 1500.0, [synth.Stage(0.0, 1.0, 101, 1)]),
        "drift": (256, 1 << 18, 2e-4, 1050.0, 1450.0, [synth.Stage(0.0, 0.5, 1001, 1)]),
        "pmps": (96, 1 << 23, 2.5e-4, 1230.0, 1518.0, synth.stages_from_table(
            [(0.0, 200.0, 0.5, 1), (200.0, 600.0, 1.0, 2), (600.0, 2000.0, 5.0, 4)], True)),
    }
    nchan, nsamp, ts, lo, hi, stages = shapes[wl]
    fch0, foff = synth.band(lo, hi, nchan)
    desc = L.FilDesc(nchan, nsamp, ts, fch0, foff, 8 if wl != "pmps" else 1)
    p = L.Plan(desc, stages)
    op = OP.Plan(nchan, nsamp, ts, fch0, foff, stages)
    np.testing.assert_array_equal(p.dms(), op.dms)
    np.testing.assert_array_equal(p.delays(), op.delays)
    assert p.max_delay == op.max_delay
    for i in (0, p.ndm // 2, p.ndm - 1):
        t = p.trial(i)
        nv, nfft = op.nv_nfft(i)
        assert (t["nv"], t["nfft"], t["ds"]) == (nv, nfft, int(op.ds_of[i]))


@pytest.mark.parametrize("wl,sub", [("drift", (16, 16)), ("drift", (256, 4)), ("pmps", (8, 24)),
                                    ("small", (1, 1)), ("small", (4, 7))])
def test_subband_plan_tables_bit_exact(L, wl, sub):
    shapes = {
        "small": (64, 1 << 16, 2e-4, 1500.0, 1200.0, [synth.Stage(0.0, 1.0, 101, 1)]),
        "drift": (256, 1 << 18, 2e-4, 1050.0, 1450.0, [synth.Stage(0.0, 0.5, 1001, 1)]),
        "pmps": (96, 1 << 23, 2.5e-4, 1230.0, 1518.0, synth.stages_from_table(
            [(0.0, 200.0, 0.5, 1), (200.0, 600.0, 1.0, 2), (600.0, 2000.0, 5.0, 4)], True)),
    }
    nchan, nsamp, ts, lo, hi, stages = shapes[wl]
    fch0, foff = synth.band(lo, hi, nchan)
    if wl == "small":
        foff = -abs(foff)  # descending band
        fch0 = 1500.0
    desc = L.FilDesc(nchan, nsamp, ts, fch0, foff, 8 if wl != "pmps" else 1)
    p = L.Plan(desc, stages, subband=sub)
    op = OP.Plan(nchan, nsamp, ts, fch0, foff, stages, subband=sub)
    info = p.subband_info()
    assert (info["nsub"], info["group"]) == sub
    np.testing.assert_array_equal(info["group_dm"], op.sub.grp_dm)
    np.testing.assert_array_equal(info["chan_delays"], op.sub.e)
    np.testing.assert_array_equal(info["sub_delays"], op.sub.D)
    np.testing.assert_array_equal(p.delays(), op.delays)
    assert p.max_delay == op.max_delay
    for i in (0, p.ndm // 2, p.ndm - 1):
        t = p.trial(i)
        nv, nfft = op.nv_nfft(i)
        assert (t["nv"], t["nfft"], t["ds"]) == (nv, nfft, int(op.ds_of[i]))
    # an exact plan reports no subbands
    assert L.Plan(desc, stages).subband_info()["nsub"] == 0


def test_subband_plan_rejects_bad_input(L):
    desc = L.FilDesc(64, 1 << 14, 2e-4, 1202.34375, 4.6875)
    for sub in ((6, 4), (0, 4), (8, 0), (8, 2000)):
        with pytest.raises(L.PssError) as e:
            L.Plan(desc, [synth.Stage(0.0, 1.0, 10, 1)], subband=sub)
        assert e.value.status == L.PSS_EINVAL


def test_plan_rejects_bad_input(L):
    desc = L.FilDesc(64, 1000, 2e-4, 1202.34375, 4.6875)
    with pytest.raises(L.PssError) as e:
        L.Plan(desc, [synth.Stage(0.0, 1.0, 2000, 1)])  # delays exceed the file
    assert e.value.status == L.PSS_EINVAL
    with pytest.raises(L.PssError):
        L.Plan(desc, [synth.Stage(0.0, 1.0, 10, 3)])     # ds not a power of two
    with pytest.raises(L.PssError):
        L.Plan(desc, [synth.Stage(0.0, 1.0, 0, 1)])      # empty stage


def test_sigma_and_threshold_match_oracle(L):
    for n in (1, 2, 4, 8, 16, 32):
        # (S well below n gives p ~ 1, where log Q itself cancels; no detection lives there)
        for S in (1.0, 8.0, 25.0, 60.0, 300.0, 2000.0, 12000.0):
            if S < 2 * n + 5:
                continue
            a = L.pss_sigma_of_power(n, S)
            b = OST.sigma_of(n, S)
            assert abs(a - b) <= 1e-9 * max(1.0, abs(b)), (n, S, a, b)
        assert abs(L.pss_power_threshold(n, 6.0) - OST.power_threshold(n, 6.0)) < 1e-8


def _random_raw(rng, ndm, per_dm, nfft, nz):
    rows = []
    for d in range(ndm):
        for _ in range(per_dm):
            n = int(2 ** rng.integers(0, 4))
            h = int(rng.integers(0, 400))
            j = int(rng.integers(0, nz))
            rows.append((d, n, h, j, np.float32(rng.uniform(20, 80)), 0))
    return np.array(rows, dtype=[("dm_idx", "<i4"), ("numharm", "<i4"), ("h", "<i4"), ("j", "<i4"),
                                 ("power", "<f4"), ("reserved", "<i4")])


@pytest.mark.parametrize("zmax,min_hits,dz", [(0, 1, 2.0), (20, 1, 2.0), (20, 2, 2.0), (6, 1, 0.3)])
def test_sift_matches_oracle(L, zmax, min_hits, dz):
    rng = np.random.default_rng(zmax + min_hits)
    nchan, nsamp = 64, 1 << 14
    fch0, foff = synth.band(1200.0, 1500.0, nchan)
    stages = [synth.Stage(0.0, 1.0, 12, 1)]
    desc = L.FilDesc(nchan, nsamp, 2e-4, fch0, foff)
    p = L.Plan(desc, stages)
    op = OP.Plan(nchan, nsamp, 2e-4, fch0, foff, stages)
    nz = int(round(2 * zmax / dz)) + 1 if zmax else 1
    Z = int(round(zmax / dz))
    raw = _random_raw(rng, 12, 40, 8192, nz)
    cfg = L.search_cfg(zmax=zmax, dz=dz, numharm=8, min_dm_hits=min_hits)
    got = L.pss_sift(p, cfg, raw)
    by_dm = {}
    for c in raw:
        n, h, j = int(c["numharm"]), int(c["h"]), int(c["j"])
        r, z = OS.fundamental(n, h, j, Z, dz)
        by_dm.setdefault(int(c["dm_idx"]), []).append(dict(
            dm_idx=int(c["dm_idx"]), numharm=n, h=h, j=j, r=r, z=z, zq=OS.zq(n, j, Z), power=float(c["power"]),
            sigma=OST.sigma_of(n, float(c["power"]))))
    ref = OS.sift(by_dm, dz, min_hits)
    assert len(got) == len(ref)
    for g, r in zip(got, ref):
        assert (int(g["dm_idx"]), int(g["numharm"]), int(g["h"]), int(g["j"]), int(g["dm_hits"])) == \
               (r["dm_idx"], r["numharm"], r["h"], r["j"], r["dm_hits"])
        assert g["r"] == r["r"] and g["z"] == r["z"]
        assert abs(g["sigma"] - r["sigma"]) < 1e-9 * r["sigma"]
        assert g["dm"] == op.dms[r["dm_idx"]]
        assert abs(g["f_hz"] - r["r"] / op.t_span(r["dm_idx"])) < 1e-12 * g["f_hz"] + 1e-15


@pytest.mark.parametrize("zmax,min_hits,dz", [(0, 2, 2.0), (20, 1, 2.0), (6, 3, 0.3)])
def test_sift_ties_and_long_chains_match_oracle(L, zmax, min_hits, dz):
    # three distinct powers make exact sigma ties between members of one group
    # (representative by lower n, then r, z, DM), and h in [0, 60) chains most
    # detections into a few long groups spanning many bins and every DM
    rng = np.random.default_rng(7 + zmax)
    nchan, nsamp, ndm = 64, 1 << 14, 10
    fch0, foff = synth.band(1200.0, 1500.0, nchan)
    stages = [synth.Stage(0.0, 1.0, ndm, 1)]
    p = L.Plan(L.FilDesc(nchan, nsamp, 2e-4, fch0, foff), stages)
    nz = int(round(2 * zmax / dz)) + 1 if zmax else 1
    Z = int(round(zmax / dz))
    raw = _random_raw(rng, ndm, 60, 8192, nz)
    raw["h"] = rng.integers(0, 60, len(raw))
    raw["power"] = rng.choice(np.array([30.0, 45.0, 60.0], np.float32), len(raw))
    raw = raw[rng.permutation(len(raw))]
    cfg = L.search_cfg(zmax=zmax, dz=dz, numharm=8, min_dm_hits=min_hits)
    got = L.pss_sift(p, cfg, raw)
    by_dm = {}
    for c in raw:
        n, h, j = int(c["numharm"]), int(c["h"]), int(c["j"])
        r, z = OS.fundamental(n, h, j, Z, dz)
        by_dm.setdefault(int(c["dm_idx"]), []).append(dict(
            dm_idx=int(c["dm_idx"]), numharm=n, h=h, j=j, r=r, z=z, zq=OS.zq(n, j, Z), power=float(c["power"]),
            sigma=OST.sigma_of(n, float(c["power"]))))
    ref = OS.sift(by_dm, dz, min_hits)
    assert 0 < len(ref) < len(raw) // 10
    assert [(int(g["dm_idx"]), int(g["numharm"]), int(g["h"]), int(g["j"]), int(g["dm_hits"])) for g in got] == \
           [(r["dm_idx"], r["numharm"], r["h"], r["j"], r["dm_hits"]) for r in ref]


@pytest.mark.parametrize("zmax,min_hits,dz", [(0, 1, 2.0), (0, 3, 2.0), (20, 1, 2.0), (20, 2, 2.0), (6, 2, 0.3)])
def test_sift_in_batches_equals_one_pass(L, zmax, min_hits, dz):
    # the pipelined search's host sift (trials sifted batch by batch, survivors merged in r order
    # for zmax 0 or linked batch by batch for zmax > 0, across-trial step at the end) gives the
    # one-pass sift's list, whatever the arrival order; dense lists make many groups span batches
    rng = np.random.default_rng(100 + zmax + min_hits)
    nchan, nsamp, ndm = 64, 1 << 14, 40
    fch0, foff = synth.band(1200.0, 1500.0, nchan)
    p = L.Plan(L.FilDesc(nchan, nsamp, 2e-4, fch0, foff), [synth.Stage(0.0, 1.0, ndm, 1)])
    nz = int(round(2 * zmax / dz)) + 1 if zmax else 1
    raw = _random_raw(rng, ndm, 120, 8192, nz)
    raw = raw[rng.permutation(len(raw))]
    cfg = L.search_cfg(zmax=zmax, dz=dz, numharm=8, min_dm_hits=min_hits)
    ref = L.pss_sift(p, cfg, raw)
    assert len(ref) > 0
    for bounds in ([0, ndm], [0, 12, 24, 36, ndm], [0, 1, 5, 5, 30, ndm]):
        got = L.pss_sift_in_batches(p, cfg, raw, bounds)
        assert got.tobytes() == ref.tobytes(), bounds
    # detections outside every batch are left out
    part = L.pss_sift_in_batches(p, cfg, raw, [0, 20])
    assert part.tobytes() == L.pss_sift(p, cfg, raw[raw["dm_idx"] < 20]).tobytes()
    with pytest.raises(L.PssError):
        L.pss_sift_in_batches(p, cfg, raw, [10, 5])


@pytest.mark.parametrize("fch0,foff,nchan,ts,lo,hi,tres,dsmax", [
    (1231.5, 3.0, 96, 250e-6, 0.0, 3896.0, 0.0, 1024),
    (290.125, 0.25, 200, 100e-6, 0.0, 784.4, 0.8e-3, 128),
    (1450.0, -1.5625, 256, 2e-4, 3.0, 500.0, 0.0, 1024),
    (1050.78125, 1.5625, 256, 2e-4, 0.0, 1.0, 1e-3, 4)])
def test_auto_plan_matches_oracle(L, fch0, foff, nchan, ts, lo, hi, tres, dsmax):
    from oracle import ddplan as ODP
    desc = L.FilDesc(nchan, 1 << 20, ts, fch0, foff)
    got = L.pss_dd_plan_auto(desc, lo, hi, tres, dsmax)
    ref = ODP.auto_plan(fch0, foff, nchan, ts, lo, hi, tres=tres, ds_max=dsmax)
    assert got == [(float(a), float(b), int(c), int(d)) for a, b, c, d in ref]


def test_auto_plan_rejects_bad_input(L):
    desc = L.FilDesc(64, 1 << 16, 2e-4, 1200.0, 4.6875)
    for args in ((10.0, 5.0, 0.0, 8), (-1.0, 5.0, 0.0, 8), (0.0, 5.0, 0.0, 3), (0.0, 5.0, 0.0, 2048)):
        with pytest.raises(L.PssError) as e:
            L.pss_dd_plan_auto(desc, *args)
        assert e.value.status == L.PSS_EINVAL
