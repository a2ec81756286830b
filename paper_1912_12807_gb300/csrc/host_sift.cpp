// Candidate sifting (paper Sect. 2 step 5, ACCEL_sift), host side.
//
// Each raw point (n, h, j) is moved to its fundamental r = h / (2n) bins,
// z = (j - Z) dz / n.  Within one DM trial, points closer than 1 bin in r
// and dz in z are linked (single linkage) and each linked group keeps its
// highest-sigma member; the survivors of all trials are linked again the
// same way, one member is kept per group and the number of distinct DM
// trials in the group is recorded.  Ties in sigma go to lower n, lower r,
// lower z, lower DM index.  Output is sorted by (DM index, n, r, z).
#include <math.h>

#include <stdint.h>
#include <stdlib.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "pss_internal.h"

namespace pss {

namespace {

struct Item {
    int32_t dm_idx, n, h, j;
    float power;
    double r, z;
    double logp;   // log Q(n, S); NAN until evaluated
    double sigma;  // -Phi^-1(Q); < 0 until evaluated
    int64_t kr, kz;  // exact link coordinates: 64 r and 32 z / dz
};

double item_logp(Item& x) {
    if (x.logp != x.logp) x.logp = log_q(x.n, (double)x.power);
    return x.logp;
}
double item_sigma(Item& x) {
    if (x.sigma < 0) x.sigma = sigma_of_power(x.n, (double)x.power);
    return x.sigma;
}

int find_root(std::vector<int>& par, int i) {
    while (par[i] != i) {
        par[i] = par[par[i]];
        i = par[i];
    }
    return i;
}

bool rep_less(const Item& a, const Item& b) {
    if (a.sigma != b.sigma) return a.sigma > b.sigma;
    if (a.n != b.n) return a.n < b.n;
    if (a.r != b.r) return a.r < b.r;
    if (a.z != b.z) return a.z < b.z;
    return a.dm_idx < b.dm_idx;
}

// Group indices [0, items.size()) by single linkage: i and j are linked
// when |r_i - r_j| <= 1 and |z_i - z_j| <= dz.  The test runs on exact
// integers: kr = 64 r = h (32/n) and kz = 32 z / dz = (j - Z)(32/n), so the
// conditions are |dkr| <= 64 and |dkz| <= 32.  Items are bucketed into cells
// of 64 x 32 units: two items of one cell always link, so a cell is one
// union-find node, and only the 4 forward-neighbouring cells need pair tests
// (skipped when their bounding boxes are too far apart or they are already
// joined).
struct Cell {
    int64_t cr, cz;
    int begin, end;  // range in the sorted order
    int64_t r_lo, r_hi, z_lo, z_hi;
};

// Flattened groups: members of group g are order[start[g] .. start[g+1]).
struct Groups {
    std::vector<int> start, members;
    int count() const { return (int)start.size() - 1; }
};

Groups link_groups(const std::vector<Item>& it, double /*dz*/) {
    const int n = (int)it.size();
    bool one_row = true;
    for (int i = 1; i < n && one_row; ++i) one_row = it[i].kz == it[0].kz;
    if (one_row) {
        // all z equal (zmax = 0): sort by r; consecutive items closer than
        // one bin link, so groups are the runs of the sorted order
        Groups G;
        std::vector<uint64_t> key(n);
        for (int i = 0; i < n; ++i) key[i] = ((uint64_t)it[i].kr << 32) | (uint32_t)i;
        std::sort(key.begin(), key.end());
        G.members.resize(n);
        G.start.push_back(0);
        for (int p = 0; p < n; ++p) {
            G.members[p] = (int)(key[p] & 0xFFFFFFFFu);
            if (p > 0 && (int64_t)(key[p] >> 32) - (int64_t)(key[p - 1] >> 32) > 64) G.start.push_back(p);
        }
        G.start.push_back(n);
        if (n == 0) G.start.resize(1);
        return G;
    }
    auto fdiv = [](int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::vector<int64_t> cr(n), cz(n);
    for (int i = 0; i < n; ++i) {
        cr[i] = fdiv(it[i].kr, 64);
        cz[i] = fdiv(it[i].kz, 32);
    }
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        if (cr[a] != cr[b]) return cr[a] < cr[b];
        if (cz[a] != cz[b]) return cz[a] < cz[b];
        return a < b;
    });
    std::vector<Cell> cells;
    for (int p = 0; p < n;) {
        int q = p;
        Cell c{cr[order[p]], cz[order[p]], p, p, INT64_MAX, INT64_MIN, INT64_MAX, INT64_MIN};
        while (q < n && cr[order[q]] == c.cr && cz[order[q]] == c.cz) {
            const Item& x = it[order[q]];
            c.r_lo = std::min(c.r_lo, x.kr);
            c.r_hi = std::max(c.r_hi, x.kr);
            c.z_lo = std::min(c.z_lo, x.kz);
            c.z_hi = std::max(c.z_hi, x.kz);
            ++q;
        }
        c.end = q;
        cells.push_back(c);
        p = q;
    }
    const int nc = (int)cells.size();
    std::vector<int> par(nc);
    std::iota(par.begin(), par.end(), 0);
    auto find_cell = [&](int64_t r, int64_t z) -> int {
        int lo = 0, hi = nc;
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (cells[mid].cr < r || (cells[mid].cr == r && cells[mid].cz < z)) lo = mid + 1;
            else hi = mid;
        }
        return (lo < nc && cells[lo].cr == r && cells[lo].cz == z) ? lo : -1;
    };
    const int64_t nb[4][2] = {{0, 1}, {1, -1}, {1, 0}, {1, 1}};
    for (int a = 0; a < nc; ++a) {
        const Cell& A = cells[a];
        for (auto& d : nb) {
            const int b = find_cell(A.cr + d[0], A.cz + d[1]);
            if (b < 0) continue;
            const Cell& B = cells[b];
            if (find_root(par, a) == find_root(par, b)) continue;
            // bounding-box gap larger than the link distance: no pair can link
            if (B.r_lo - A.r_hi > 64 || A.r_lo - B.r_hi > 64 || B.z_lo - A.z_hi > 32 || A.z_lo - B.z_hi > 32)
                continue;
            bool linked = false;
            for (int p = A.begin; p < A.end && !linked; ++p) {
                const Item& x = it[order[p]];
                for (int q = B.begin; q < B.end; ++q) {
                    const Item& y = it[order[q]];
                    if (std::llabs(x.kr - y.kr) <= 64 && std::llabs(x.kz - y.kz) <= 32) {
                        linked = true;
                        break;
                    }
                }
            }
            if (linked) {
                const int ra = find_root(par, a), rb = find_root(par, b);
                par[std::max(ra, rb)] = std::min(ra, rb);
            }
        }
    }
    // roots in order of first appearance; counting sort of cells by root
    std::vector<int> slot(nc, -1), cnt;
    int ng = 0;
    for (int c = 0; c < nc; ++c) {
        const int r = find_root(par, c);
        if (slot[r] < 0) {
            slot[r] = ng++;
            cnt.push_back(0);
        }
        cnt[slot[r]] += cells[c].end - cells[c].begin;
    }
    Groups G;
    G.start.assign(ng + 1, 0);
    for (int g = 0; g < ng; ++g) G.start[g + 1] = G.start[g] + cnt[g];
    G.members.resize(n);
    std::vector<int> fill(G.start.begin(), G.start.end() - 1);
    for (int c = 0; c < nc; ++c) {
        const int g = slot[find_root(par, c)];
        for (int p = cells[c].begin; p < cells[c].end; ++p) G.members[fill[g]++] = order[p];
    }
    return G;
}

// Representative of a linked group: the highest sigma (ties: lower n, r, z,
// DM index).  sigma is strictly increasing in S for a fixed n, so only the
// largest-S member of each harmonic stage can win.  sigma is a decreasing
// function of log Q, so those few members are ranked by log Q; sigma itself
// is evaluated only where two log Q values are too close (1e-12 relative) for
// their order to decide the order of the sigmas, and for the winner.
int pick_rep(std::vector<Item>& items, const int* mem, int nm) {
    int best_of_n[8];
    for (int i = 0; i < 8; ++i) best_of_n[i] = -1;
    for (int q = 0; q < nm; ++q) {
        const int k = mem[q];
        const Item& a = items[k];
        int li = 0;
        while ((1 << li) < a.n && li < 7) ++li;
        int& b = best_of_n[li];
        if (b < 0) {
            b = k;
            continue;
        }
        const Item& c = items[b];
        if (a.power > c.power || (a.power == c.power && (a.r < c.r || (a.r == c.r && (a.z < c.z || (a.z == c.z && a.dm_idx < c.dm_idx))))))
            b = k;
    }
    int best = -1;
    for (int i = 0; i < 8; ++i) {
        const int k = best_of_n[i];
        if (k < 0) continue;
        if (best < 0) {
            best = k;
            continue;
        }
        const double lk = item_logp(items[k]), lb = item_logp(items[best]);
        if (fabs(lk - lb) > 1e-12 * std::max(fabs(lk), fabs(lb))) {
            if (lk < lb) best = k;
        } else {
            item_sigma(items[k]);
            item_sigma(items[best]);
            if (rep_less(items[k], items[best])) best = k;
        }
    }
    item_sigma(items[best]);
    return best;
}

}  // namespace

void bucket_by_dm(const pss_raw_cand* raw, int64_t n, int64_t ndm, std::vector<int64_t>* order,
                  std::vector<std::pair<int64_t, int64_t>>* buckets) {
    std::vector<int64_t> cnt((size_t)ndm + 1, 0);
    for (int64_t i = 0; i < n; ++i) cnt[(size_t)raw[i].dm_idx + 1]++;
    for (int64_t d = 0; d < ndm; ++d) cnt[(size_t)d + 1] += cnt[(size_t)d];
    order->assign((size_t)n, 0);
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (int64_t i = 0; i < n; ++i) (*order)[(size_t)pos[(size_t)raw[i].dm_idx]++] = i;
    buckets->clear();
    for (int64_t d = 0; d < ndm; ++d)
        if (cnt[(size_t)d + 1] > cnt[(size_t)d]) buckets->push_back({cnt[(size_t)d], cnt[(size_t)d + 1]});
}

void sort_raw(std::vector<pss_raw_cand>* v, int64_t ndm) {
    std::vector<int64_t> order;
    std::vector<std::pair<int64_t, int64_t>> bk;
    bucket_by_dm(v->data(), (int64_t)v->size(), ndm, &order, &bk);
    std::vector<pss_raw_cand> out(v->size());
    for (size_t i = 0; i < order.size(); ++i) out[i] = (*v)[(size_t)order[i]];
    parallel_for((int64_t)bk.size(), 8, [&](int64_t b) {
        std::sort(out.begin() + bk[(size_t)b].first, out.begin() + bk[(size_t)b].second,
                  [](const pss_raw_cand& x, const pss_raw_cand& y) {
                      if (x.numharm != y.numharm) return x.numharm < y.numharm;
                      if (x.j != y.j) return x.j < y.j;
                      return x.h < y.h;
                  });
    });
    v->swap(out);
}

pss_status sift(const Plan& P, const pss_search_cfg& cfg, const pss_raw_cand* raw, int64_t n,
                std::vector<pss_cand>* out) {
    out->clear();
    const int Z = cfg.zmax ? (int)llround(cfg.zmax / cfg.dz) : 0;
    const double dz = cfg.dz;
    for (int64_t i = 0; i < n; ++i) {
        if (raw[i].dm_idx < 0 || raw[i].dm_idx >= P.ndm()) return fail(PSS_EINVAL, "pss_sift: dm_idx out of range");
        if (raw[i].numharm < 1 || raw[i].numharm > 32 || (raw[i].numharm & (raw[i].numharm - 1))) return fail(PSS_EINVAL, "pss_sift: numharm must be a power of two in [1, 32]");
    }
    std::vector<int64_t> order;
    std::vector<std::pair<int64_t, int64_t>> bk;
    bucket_by_dm(raw, n, P.ndm(), &order, &bk);
    // within each DM trial (independent: in parallel)
    std::vector<std::vector<Item>> surv(bk.size());
    parallel_for((int64_t)bk.size(), 4, [&](int64_t b) {
        std::vector<Item> items;
        items.reserve((size_t)(bk[(size_t)b].second - bk[(size_t)b].first));
        for (int64_t q = bk[(size_t)b].first; q < bk[(size_t)b].second; ++q) {
            const pss_raw_cand& c = raw[order[(size_t)q]];
            Item it;
            it.dm_idx = c.dm_idx;
            it.n = c.numharm;
            it.h = c.h;
            it.j = c.j;
            it.power = c.power;
            it.r = (double)c.h / (double)(2 * c.numharm);
            it.z = (double)(c.j - Z) * dz / (double)c.numharm;
            it.sigma = -1.0;  // evaluated on demand by pick_rep
            it.logp = NAN;
            it.kr = (int64_t)c.h * (32 / c.numharm);
            it.kz = (int64_t)(c.j - Z) * (32 / c.numharm);
            items.push_back(it);
        }
        const Groups G = link_groups(items, dz);
        for (int g = 0; g < G.count(); ++g)
            surv[(size_t)b].push_back(
                items[pick_rep(items, G.members.data() + G.start[g], G.start[g + 1] - G.start[g])]);
    });
    std::vector<Item> survivors;
    for (auto& v : surv) survivors.insert(survivors.end(), v.begin(), v.end());

    // across DM trials
    const Groups G = link_groups(survivors, dz);
    for (int g = 0; g < G.count(); ++g) {
        const int* mem = G.members.data() + G.start[g];
        const int nm = G.start[g + 1] - G.start[g];
        const int best = pick_rep(survivors, mem, nm);
        std::vector<int32_t> dms;
        for (int q = 0; q < nm; ++q) dms.push_back(survivors[mem[q]].dm_idx);
        std::sort(dms.begin(), dms.end());
        int hits = (int)(std::unique(dms.begin(), dms.end()) - dms.begin());
        if (hits < cfg.min_dm_hits) continue;
        const Item& b = survivors[best];
        pss_cand c;
        c.dm_idx = b.dm_idx;
        c.numharm = b.n;
        c.dm = P.dms[b.dm_idx];
        c.r = b.r;
        c.z = b.z;
        c.f_hz = b.r / P.t_span(b.dm_idx);
        c.sigma = b.sigma;
        c.power = b.power;
        c.dm_hits = hits;
        c.h = b.h;
        c.j = b.j;
        out->push_back(c);
    }
    std::sort(out->begin(), out->end(), [](const pss_cand& a, const pss_cand& b) {
        if (a.dm_idx != b.dm_idx) return a.dm_idx < b.dm_idx;
        if (a.numharm != b.numharm) return a.numharm < b.numharm;
        if (a.r != b.r) return a.r < b.r;
        return a.z < b.z;
    });
    return PSS_OK;
}

}  // namespace pss
