"""Pins for candidate sifting (Sect. 2 step 5) against brute force.

The oracle groups candidates by a sorted scan over r with an early break and
a union-find.  These tests rebuild the same partition from its definition:
the graph whose edges join every pair with |dr| <= 1 bin and |dz| <= dz
(all pairs, no ordering), split into connected components by scipy's
library routine.  Inputs sit on exact 1/8-bin and dz grids, so pairs exactly
at the linking limits occur often and a strict/non-strict slip shows.
"""
from fractions import Fraction

import numpy as np
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

from oracle import sift as SF

DZ = 2.0
Z = 8


def _cand(uid, dm, n, h, j, sigma):
    r, z = SF.fundamental(n, h, j, Z, DZ)
    return dict(uid=uid, dm_idx=dm, numharm=n, h=h, j=j, r=r, z=z,
                zq=SF.zq(n, j, Z), sigma=sigma, power=0.0)


def _random_cands(rng, n_dm, per_dm):
    out, uid = [], 0
    sig = rng.permutation(n_dm * per_dm).astype(float) / 7.0 + 5.0   # distinct sigmas
    for dm in range(n_dm):
        for _ in range(per_dm):
            n = int(rng.choice([1, 2, 4]))
            h = int(rng.integers(0, 8 * n * 6))           # r = h / (2n) in [0, 24) on a 1/8 grid
            j = Z + int(rng.integers(-3 * n, 3 * n + 1))  # z / dz in [-3, 3] on a 1/n grid
            out.append(_cand(uid, dm, n, h, j, float(sig[uid])))
            uid += 1
    return out


def _components(cands):
    """Connected components of the all-pairs link graph, as sets of uids."""
    m = len(cands)
    if m == 0:
        return []
    rq = [Fraction(c["h"], 2 * c["numharm"]) for c in cands]
    zq = [c["zq"] for c in cands]
    rows, cols = [], []
    for a in range(m):
        for b in range(m):
            if abs(rq[a] - rq[b]) <= 1 and abs(zq[a] - zq[b]) <= 1:
                rows.append(a)
                cols.append(b)
    g = csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(m, m))
    k, lab = connected_components(g, directed=False)
    comps = [set() for _ in range(k)]
    for i, l in enumerate(lab):
        comps[l].add(i)
    return comps


def _brute_within(cands):
    return {max((cands[i] for i in comp), key=lambda c: c["sigma"])["uid"]
            for comp in _components(cands)}


def _brute_across(cands, min_dm_hits):
    out = []
    for comp in _components(cands):
        rep = max((cands[i] for i in comp), key=lambda c: c["sigma"])
        hits = len({cands[i]["dm_idx"] for i in comp})
        if hits >= min_dm_hits:
            out.append((rep["uid"], hits))
    return out


def test_link_limits_are_inclusive():
    # exactly 1 bin apart in r links; 1 + 1/8 does not
    a = _cand(0, 0, 1, 20, Z, 9.0)          # r = 10
    b = _cand(1, 0, 1, 22, Z, 8.0)          # r = 11
    c = _cand(2, 0, 4, 97, Z, 7.0)          # r = 12.125
    assert sorted(x["uid"] for x in SF.sift_within([a, b, c], DZ)) == [0, 2]
    # exactly one dz step apart in z links; a z/dz gap of 5/4 does not
    d = _cand(3, 0, 1, 40, Z + 1, 9.0)      # r = 20, z/dz = 1
    e = _cand(4, 0, 2, 80, Z + 4, 8.0)      # r = 20, z/dz = 2
    f = _cand(5, 0, 4, 160, Z + 13, 7.0)    # r = 20, z/dz = 13/4
    assert sorted(x["uid"] for x in SF.sift_within([d, e, f], DZ)) == [3, 5]
    # single linkage: the chain d - e links d to a member 2 steps away
    g = _cand(6, 0, 1, 40, Z + 3, 6.0)      # z/dz = 3, 1 step from e only
    assert sorted(x["uid"] for x in SF.sift_within([d, e, g], DZ)) == [3]


def test_sift_within_equals_components_of_all_pairs_graph():
    rng = np.random.default_rng(5)
    for trial in range(40):
        cands = _random_cands(rng, 1, int(rng.integers(0, 60)))
        got = {c["uid"] for c in SF.sift_within(cands, DZ)}
        assert got == _brute_within(cands), trial


def test_sift_across_equals_components_with_dm_hits():
    rng = np.random.default_rng(6)
    for trial in range(30):
        cands = _random_cands(rng, 5, int(rng.integers(1, 25)))
        for min_hits in (1, 2, 3):
            got = SF.sift_across(cands, DZ, min_hits)
            want = _brute_across(cands, min_hits)
            assert sorted((c["uid"], c["dm_hits"]) for c in got) == sorted(want), (trial, min_hits)
            keys = [(c["dm_idx"], c["numharm"], c["r"], c["z"]) for c in got]
            assert keys == sorted(keys)


def test_sift_is_within_then_across():
    rng = np.random.default_rng(7)
    for trial in range(20):
        cands = _random_cands(rng, 4, int(rng.integers(1, 30)))
        by_dm = {}
        for c in cands:
            by_dm.setdefault(c["dm_idx"], []).append(c)
        survivors = []
        for dm in sorted(by_dm):
            keep = _brute_within(by_dm[dm])
            survivors.extend(c for c in by_dm[dm] if c["uid"] in keep)
        want = _brute_across(survivors, 2)
        got = SF.sift(by_dm, DZ, 2)
        assert sorted((c["uid"], c["dm_hits"]) for c in got) == sorted(want), trial


def test_float_path_matches_exact_path():
    # candidates without (h, j) are linked on their binary-exact floats
    rng = np.random.default_rng(8)
    cands = _random_cands(rng, 1, 50)
    bare = [{k: v for k, v in c.items() if k not in ("zq",)} for c in cands]
    assert ({c["uid"] for c in SF.sift_within(bare, DZ)}
            == {c["uid"] for c in SF.sift_within(cands, DZ)})
    # both forms in one call: the exact (r, z/dz) must be the same point as the float one
    mixed = [bare[i] if i % 2 else cands[i] for i in range(len(cands))]
    assert ({c["uid"] for c in SF.sift_within(mixed, DZ)}
            == {c["uid"] for c in SF.sift_within(cands, DZ)})
    for n in (1, 2, 4, 8):
        for j in range(0, 2 * Z + 1):
            assert SF.zq(n, j, Z) * Fraction(DZ) == Fraction(SF.fundamental(n, 3, j, Z, DZ)[1])
