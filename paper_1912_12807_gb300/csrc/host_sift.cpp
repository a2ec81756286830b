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

}  // namespace

pss_status sift(const Plan& P, const pss_search_cfg& cfg, const pss_raw_cand* raw, int64_t n,
                std::vector<pss_cand>* out) {
    out->clear();
    const int Z = cfg.zmax ? (int)llround(cfg.zmax / cfg.dz) : 0;
    const double dz = cfg.dz;
    // bucket by DM trial
    std::vector<int64_t> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return raw[a].dm_idx < raw[b].dm_idx; });
    std::vector<Item> survivors;
    int64_t p = 0;
    while (p < n) {
        int64_t q = p;
        const int32_t dm = raw[idx[p]].dm_idx;
        if (dm < 0 || dm >= P.ndm()) return fail(PSS_EINVAL, "pss_sift: dm_idx out of range");
        std::vector<Item> items;
        while (q < n && raw[idx[q]].dm_idx == dm) {
            const pss_raw_cand& c = raw[idx[q]];
            if (c.numharm < 1) return fail(PSS_EINVAL, "pss_sift: numharm < 1");
            Item it;
            it.dm_idx = c.dm_idx;
            it.n = c.numharm;
            it.h = c.h;
            it.j = c.j;
            it.power = c.power;
            it.r = (double)c.h / (double)(2 * c.numharm);
            it.z = (double)(c.j - Z) * dz / (double)c.numharm;
            it.sigma = sigma_of_power(c.numharm, (double)c.power);
            items.push_back(it);
            ++q;
        }
        for (auto& g : link_groups(items, dz)) {
            int best = g[0];
            for (int k : g)
                if (rep_less(items[k], items[best])) best = k;
            survivors.push_back(items[best]);
        }
        p = q;
    }
    for (auto& g : link_groups(survivors, dz)) {
        int best = g[0];
        std::vector<int32_t> dms;
        for (int k : g) {
            if (rep_less(survivors[k], survivors[best])) best = k;
            dms.push_back(survivors[k].dm_idx);
        }
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
