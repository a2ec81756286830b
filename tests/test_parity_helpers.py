"""The point-wise parity helpers (tests/_parity.py) against the whole-plane
oracle on small inputs: the plane evaluated point by point equals the
plane rows of the definition, and the candidate check accepts the oracle's
own raw candidates and rejects moved or altered ones."""
import numpy as np
import pytest

from oracle import harmsum as OH
from oracle import response as OR
from oracle import stats as OST

from _parity import check_candidates_at_points, oracle_plane_points


def _spectrum(M, seed, tone_bin=None, tone_amp=0.0):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) / np.sqrt(2.0)
    if tone_bin is not None:
        A[tone_bin] += tone_amp
    return A


@pytest.mark.parametrize("zmax,dz", [(0, 2.0), (6, 2.0), (5, 0.5)])
def test_points_equal_plane_rows(zmax, dz):
    M = 1024
    Ap = _spectrum(M, 3)
    plane = OR.power_plane(Ap, zmax, dz, 16, "direct")
    nz, H = plane.shape
    rng = np.random.default_rng(4)
    js = rng.integers(0, nz, 600)
    hs = np.concatenate([rng.integers(0, H, 590), [0, 1, 2, H - 1, H - 2, H - 3, 31, 32, 33, 34]])
    got = oracle_plane_points(Ap, zmax, dz, 16, js, hs)
    ref = plane[js, hs]
    assert np.max(np.abs(got - ref) / np.maximum(ref, 1.0)) < 1e-12


def _rows(cands, dm_idx=3):
    dt = np.dtype([("dm_idx", "i4"), ("numharm", "i4"), ("h", "i4"), ("j", "i4"), ("power", "f4")])
    out = np.zeros(len(cands), dtype=dt)
    for i, (n, h, j, S) in enumerate(cands):
        out[i] = (dm_idx, n, h, j, S)
    return out


def test_candidate_check_accepts_oracle_and_rejects_planted_errors():
    M, zmax, dz, numharm = 2048, 4, 2.0, 4
    Ap = _spectrum(M, 5, tone_bin=300, tone_amp=14.0)
    Ap[600] += 8.0
    plane = OR.power_plane(Ap, zmax, dz, 16, "direct")
    nz, H = plane.shape
    thr = OST.thresholds(numharm, 3.0)
    T = 1.0
    raw = OH.raw_candidates(plane, numharm, int(zmax / dz), thr, T, 1.0)
    assert len(raw) >= 3
    rows = _rows(raw)
    args = (Ap, 3, numharm, zmax, dz, 16, nz, H, T, 1.0, 3.0)
    assert check_candidates_at_points(rows, *args) == len(raw)
    # a candidate moved off its local maximum fails
    bad = rows.copy()
    bad[0]["h"] += 1
    with pytest.raises(AssertionError):
        check_candidates_at_points(bad, *args)
    # a wrong power fails
    bad = rows.copy()
    bad[0]["power"] *= 1.001
    with pytest.raises(AssertionError):
        check_candidates_at_points(bad, *args)
    # a wrong stage fails
    bad = rows.copy()
    k = int(np.argmax(bad["numharm"] == 1))
    bad[k]["numharm"] = 2
    with pytest.raises(AssertionError):
        check_candidates_at_points(bad, *args)
