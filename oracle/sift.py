"""Candidate sifting (Sect. 2 step 5, ACCEL_sift).

The paper names the step only.  Reading used here:

* Each raw candidate is moved to its fundamental: r = h / (2n) bins,
  z = (j - Z) dz / n (both exact in FP64 for power-of-two n).
* Within one DM trial, candidates are linked when |dr| <= 1 bin and
  |dz| <= dz (single linkage); each linked group keeps one representative.
* Survivors of all DM trials are linked again the same way; each group
  keeps one representative and records dm_hits, the number of distinct DM
  trials in the group; groups with dm_hits < min_dm_hits are dropped.
* The representative is the member with the highest sigma; exact ties go
  to lower n, then lower r, lower z, lower DM index.
* The final list is sorted by (DM index, n, r, z).
"""
from __future__ import annotations

from typing import Dict, List


def _find(par, i):
    while par[i] != i:
        par[i] = par[par[i]]
        i = par[i]
    return i


def _groups(items: List[Dict], dz: float) -> List[List[int]]:
    order = sorted(range(len(items)), key=lambda i: (items[i]["r"], items[i]["z"], i))
    par = list(range(len(items)))
    for a_pos, a in enumerate(order):
        ra, za = items[a]["r"], items[a]["z"]
        for b in order[a_pos + 1:]:
            if items[b]["r"] - ra > 1.0:
                break
            if abs(items[b]["z"] - za) <= dz:
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
    return float(h) / float(2 * n), float(j - Z) * dz / float(n)


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
