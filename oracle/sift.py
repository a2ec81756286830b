"""Candidate sifting (Sect. 2 step 5, ACCEL_sift).

The paper names the step only.  Reading used here:

* Each raw candidate is moved to its fundamental: r = h / (2n) bins,
  z = (j - Z) dz / n.
* Within one DM trial, candidates are linked when |dr| <= 1 bin and
  |dz| <= dz (single linkage); each linked group keeps one representative.
  Both conditions are evaluated exactly, on rationals (r = h/(2n) and
  z/dz = (j - Z)/n), not on rounded floating-point values.
* Survivors of all DM trials are linked again the same way; each group
  keeps one representative and records dm_hits, the number of distinct DM
  trials in the group; groups with dm_hits < min_dm_hits are dropped.
* The representative is the member with the highest sigma; exact ties go
  to lower n, then lower r, lower z, lower DM index.
* The final list is sorted by (DM index, n, r, z).
"""
from __future__ import annotations

from fractions import Fraction
from typing import Dict, List


def _find(par, i):
    while par[i] != i:
        par[i] = par[par[i]]
        i = par[i]
    return i


def _rz(c: Dict, dz: float):
    """Exact (r, z/dz): from (h, j, n, Z) when the candidate carries them,
    else from its (binary-exact) floats."""
    if "zq" in c:
        return Fraction(c["h"], 2 * c["numharm"]), c["zq"]
    return Fraction(c["r"]), Fraction(c["z"]) / Fraction(dz)


def _groups(items: List[Dict], dz: float) -> List[List[int]]:
    ex = [_rz(c, dz) for c in items]
    order = sorted(range(len(items)), key=lambda i: (ex[i][0], ex[i][1], i))
    par = list(range(len(items)))
    for a_pos, a in enumerate(order):
        ra, za = ex[a]
        for b in order[a_pos + 1:]:
            if ex[b][0] - ra > 1:
                break
            if abs(ex[b][1] - za) <= 1:
                pa, pb = _find(par, a), _find(par, b)
                if pa != pb:
                    par[max(pa, pb)] = min(pa, pb)
    g: Dict[int, List[int]] = {}
    for i in range(len(items)):
        g.setdefault(_find(par, i), []).append(i)
    return list(g.values())


def _rep_key(c: Dict):
    return (-c["sigma"], c["numharm"], c["r"], c["z"], c["dm_idx"])


def fundamental(n: int, h: int, j: int, Z: int, dz: float):
    """(r, z) of the fundamental as floats; zq(n, j, Z) gives z/dz exactly."""
    return float(h) / float(2 * n), float(j - Z) * dz / float(n)


def zq(n: int, j: int, Z: int) -> Fraction:
    return Fraction(j - Z, n)


def sift_within(cands: List[Dict], dz: float) -> List[Dict]:
    reps = []
    for grp in _groups(cands, dz):
        reps.append(min((cands[i] for i in grp), key=_rep_key))
    return reps


def sift_across(cands: List[Dict], dz: float, min_dm_hits: int) -> List[Dict]:
    out = []
    for grp in _groups(cands, dz):
        rep = dict(min((cands[i] for i in grp), key=_rep_key))
        rep["dm_hits"] = len({cands[i]["dm_idx"] for i in grp})
        if rep["dm_hits"] >= min_dm_hits:
            out.append(rep)
    out.sort(key=lambda c: (c["dm_idx"], c["numharm"], c["r"], c["z"]))
    return out


def sift(raw_by_dm: Dict[int, List[Dict]], dz: float, min_dm_hits: int) -> List[Dict]:
    survivors = []
    for dm_idx in sorted(raw_by_dm):
        survivors.extend(sift_within(raw_by_dm[dm_idx], dz))
    return sift_across(survivors, dz, min_dm_hits)
