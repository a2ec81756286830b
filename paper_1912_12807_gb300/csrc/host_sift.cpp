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

#include <algorithm>
#include <numeric>
#include <vector>

#include "pss_internal.h"

namespace pss {

namespace {

struct Item {
    int32_t dm_idx, n, h, j;
    float power;
    double r, z, sigma;
};

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

// Group indices [0, items.size()) by single linkage in (r, z).
std::vector<std::vector<int>> link_groups(const std::vector<Item>& it, double dz) {
    const int n = (int)it.size();
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        if (it[a].r != it[b].r) return it[a].r < it[b].r;
        if (it[a].z != it[b].z) return it[a].z < it[b].z;
        return a < b;
    });
    std::vector<int> par(n);
    std::iota(par.begin(), par.end(), 0);
    for (int p = 0; p < n; ++p) {
        const Item& a = it[order[p]];
        for (int q = p + 1; q < n; ++q) {
            const Item& b = it[order[q]];
            if (b.r - a.r > 1.0) break;
            if (fabs(b.z - a.z) <= dz) {
                int ra = find_root(par, order[p]), rb = find_root(par, order[q]);
                if (ra != rb) par[std::max(ra, rb)] = std::min(ra, rb);
            }
        }
    }
    std::vector<std::vector<int>> groups;
    std::vector<int> slot(n, -1);
    for (int i = 0; i < n; ++i) {
        int r = find_root(par, i);
        if (slot[r] < 0) {
            slot[r] = (int)groups.size();
            groups.emplace_back();
        }
        groups[slot[r]].push_back(i);
    }
    return groups;
}

// Representative of a linked group: the highest sigma (ties: lower n, r, z,
// DM index).  sigma is strictly increasing in S for a fixed n, so only the
// largest-S member of each harmonic stage can win; sigma is evaluated for
// those alone (items with sigma < 0 have not been evaluated yet).
int pick_rep(std::vector<Item>& items, const std::vector<int>& g) {
    int best_of_n[8];
    for (int i = 0; i < 8; ++i) best_of_n[i] = -1;
    for (int k : g) {
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
        if (items[k].sigma < 0) items[k].sigma = sigma_of_power(items[k].n, (double)items[k].power);
        if (best < 0 || rep_less(items[k], items[best])) best = k;
    }
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
        if (raw[i].numharm < 1 || raw[i].numharm > 64 || (raw[i].numharm & (raw[i].numharm - 1))) return fail(PSS_EINVAL, "pss_sift: numharm must be a power of two in [1, 64]");
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
            items.push_back(it);
        }
        for (auto& g : link_groups(items, dz)) surv[(size_t)b].push_back(items[pick_rep(items, g)]);
    });
    std::vector<Item> survivors;
    for (auto& v : surv) survivors.insert(survivors.end(), v.begin(), v.end());

    // across DM trials
    for (auto& g : link_groups(survivors, dz)) {
        const int best = pick_rep(survivors, g);
        std::vector<int32_t> dms;
        for (int k : g) dms.push_back(survivors[k].dm_idx);
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
