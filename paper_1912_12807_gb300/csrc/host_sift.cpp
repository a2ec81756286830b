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
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <vector>

#include "pss_internal.h"

namespace pss {

namespace {

using Item = SiftItem;

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
// joined; for the cell above or to the right the bounding boxes decide).
// Cells are found through a hash table (the same groups, in any order).
struct Cell {
    int64_t cr, cz;
    int begin, end;  // range of the cell's members in the order
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
        // one bin link, so groups are the runs of the sorted order (items
        // that arrive sorted by r, as the pipelined search keeps them, skip
        // the sort)
        Groups G;
        G.members.resize(n);
        G.start.push_back(0);
        bool sorted = true;
        for (int i = 1; i < n && sorted; ++i) sorted = it[i - 1].kr <= it[i].kr;
        if (sorted) {
            for (int p = 0; p < n; ++p) {
                G.members[p] = p;
                if (p > 0 && it[p].kr - it[p - 1].kr > 64) G.start.push_back(p);
            }
        } else {
            std::vector<uint64_t> key(n);
            for (int i = 0; i < n; ++i) key[i] = ((uint64_t)it[i].kr << 32) | (uint32_t)i;
            std::sort(key.begin(), key.end());
            for (int p = 0; p < n; ++p) {
                G.members[p] = (int)(key[p] & 0xFFFFFFFFu);
                if (p > 0 && (int64_t)(key[p] >> 32) - (int64_t)(key[p - 1] >> 32) > 64) G.start.push_back(p);
            }
        }
        G.start.push_back(n);
        if (n == 0) G.start.resize(1);
        return G;
    }
    auto fdiv = [](int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); };
    // cells in an open-addressing hash table keyed by (cell r, cell z), in order of first
    // appearance; the groups are the same sets whatever the order of the cells
    std::vector<int64_t> cr(n), cz(n);
    for (int i = 0; i < n; ++i) {
        cr[i] = fdiv(it[i].kr, 64);
        cz[i] = fdiv(it[i].kz, 32);
    }
    size_t cap = 16;
    while (cap < 2 * (size_t)n) cap <<= 1;
    std::vector<int> table(cap, -1);
    std::vector<Cell> cells;
    cells.reserve((size_t)n);
    auto hash_of = [](int64_t r, int64_t z) {
        uint64_t h = (uint64_t)r * 0x9E3779B97F4A7C15ull ^ ((uint64_t)z + 0x632BE59BD9B4E019ull) * 0xC2B2AE3D27D4EB4Full;
        return h ^ (h >> 29);
    };
    auto find_cell = [&](int64_t r, int64_t z) -> int {  // -1 if absent
        for (size_t h = hash_of(r, z) & (cap - 1);; h = (h + 1) & (cap - 1)) {
            const int c = table[h];
            if (c < 0) return -1;
            if (cells[(size_t)c].cr == r && cells[(size_t)c].cz == z) return c;
        }
    };
    std::vector<int> cell_of(n);
    for (int i = 0; i < n; ++i) {
        size_t h = hash_of(cr[i], cz[i]) & (cap - 1);
        int c;
        for (;; h = (h + 1) & (cap - 1)) {
            c = table[h];
            if (c < 0) {
                c = (int)cells.size();
                table[h] = c;
                cells.push_back(Cell{cr[i], cz[i], 0, 0, INT64_MAX, INT64_MIN, INT64_MAX, INT64_MIN});
                break;
            }
            if (cells[(size_t)c].cr == cr[i] && cells[(size_t)c].cz == cz[i]) break;
        }
        Cell& C = cells[(size_t)c];
        ++C.end;  // count for now
        C.r_lo = std::min(C.r_lo, it[i].kr);
        C.r_hi = std::max(C.r_hi, it[i].kr);
        C.z_lo = std::min(C.z_lo, it[i].kz);
        C.z_hi = std::max(C.z_hi, it[i].kz);
        cell_of[i] = c;
    }
    const int nc = (int)cells.size();
    // members of each cell contiguous in `order` (counting sort by cell)
    {
        int acc = 0;
        for (Cell& C : cells) {
            const int k = C.end;
            C.begin = acc;
            C.end = acc;
            acc += k;
        }
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[cells[(size_t)cell_of[i]].end++] = i;
    std::vector<int> par(nc);
    std::iota(par.begin(), par.end(), 0);
    // forward neighbours (cr, cz+1), (cr+1, cz-1), (cr+1, cz), (cr+1, cz+1) of every cell
    for (int a = 0; a < nc; ++a) {
        const Cell& A = cells[(size_t)a];
        const int nbr[4] = {find_cell(A.cr, A.cz + 1), find_cell(A.cr + 1, A.cz - 1), find_cell(A.cr + 1, A.cz),
                            find_cell(A.cr + 1, A.cz + 1)};
        for (int k = 0; k < 4; ++k) {
            const int b = nbr[k];
            if (b < 0) continue;
            const Cell& B = cells[(size_t)b];
            if (find_root(par, a) == find_root(par, b)) continue;
            // bounding-box gap larger than the link distance: no pair can link
            if (B.r_lo - A.r_hi > 64 || A.r_lo - B.r_hi > 64 || B.z_lo - A.z_hi > 32 || A.z_lo - B.z_hi > 32)
                continue;
            // the cell above (k = 0) or to the right (k = 2): the other coordinate differs by less
            // than a cell for every pair, so the closest pair of the gap's direction links
            bool linked = k == 0 || k == 2;
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
        cnt[slot[r]] += cells[(size_t)c].end - cells[(size_t)c].begin;
    }
    Groups G;
    G.start.assign(ng + 1, 0);
    for (int g = 0; g < ng; ++g) G.start[g + 1] = G.start[g] + cnt[g];
    G.members.resize(n);
    std::vector<int> fill(G.start.begin(), G.start.end() - 1);
    for (int c = 0; c < nc; ++c) {
        const int g = slot[find_root(par, c)];
        for (int p = cells[(size_t)c].begin; p < cells[(size_t)c].end; ++p) G.members[fill[g]++] = order[p];
    }
    return G;
}

// Representative of a linked group: the highest sigma (ties: lower n, r, z,
// DM index).  sigma is strictly increasing in S for a fixed n, so only the
// largest-S member of each harmonic stage can win.  sigma is a decreasing
// function of log Q, so those few members are ranked by log Q; sigma itself
// is evaluated only where two log Q values are too close (1e-12 relative) for
// their order to decide the order of the sigmas, and for the winner when the
// caller needs it (the final, across-trial representatives).
int pick_rep(std::vector<Item>& items, const int* mem, int nm, bool need_sigma) {
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
    if (need_sigma) item_sigma(items[best]);
    return best;
}

}  // namespace

void bucket_by_dm(const pss_raw_cand* raw, int64_t n, int64_t ndm, std::vector<int64_t>* order,
                  std::vector<std::pair<int64_t, int64_t>>* buckets) {
    // stable counting sort by DM index over contiguous chunks of the input in parallel: chunk t's
    // items of trial d follow those of chunks < t (the order of the serial counting sort)
    const int64_t T = n < (int64_t)1 << 16 ? 1 : std::min<int64_t>(16, n >> 15);
    std::vector<int64_t> cnt((size_t)(T * ndm), 0);  // [chunk][trial]
    auto lo_of = [&](int64_t t) { return t * n / T; };
    parallel_for(T, 1, [&](int64_t t) {
        int64_t* c = cnt.data() + t * ndm;
        for (int64_t i = lo_of(t); i < lo_of(t + 1); ++i) c[raw[i].dm_idx]++;
    });
    std::vector<int64_t> pos((size_t)(T * ndm));
    buckets->clear();
    int64_t acc = 0;
    for (int64_t d = 0; d < ndm; ++d) {
        const int64_t first = acc;
        for (int64_t t = 0; t < T; ++t) {
            pos[(size_t)(t * ndm + d)] = acc;
            acc += cnt[(size_t)(t * ndm + d)];
        }
        if (acc > first) buckets->push_back({first, acc});
    }
    order->resize((size_t)n);
    parallel_for(T, 1, [&](int64_t t) {
        int64_t* p = pos.data() + t * ndm;
        for (int64_t i = lo_of(t); i < lo_of(t + 1); ++i) (*order)[(size_t)p[raw[i].dm_idx]++] = i;
    });
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

pss_status sift_within(const Plan& P, const pss_search_cfg& cfg, const pss_raw_cand* raw, int64_t n,
                       std::vector<SiftItem>* out) {
    const int Z = cfg.zmax ? (int)llround(cfg.zmax / cfg.dz) : 0;
    const double dz = cfg.dz;
    for (int64_t i = 0; i < n; ++i) {
        if (raw[i].dm_idx < 0 || raw[i].dm_idx >= P.ndm()) return fail(PSS_EINVAL, "pss_sift: dm_idx out of range");
        if (raw[i].numharm < 1 || raw[i].numharm > 32 || (raw[i].numharm & (raw[i].numharm - 1))) return fail(PSS_EINVAL, "pss_sift: numharm must be a power of two in [1, 32]");
    }
    const bool dbg = getenv("PSS_TIMING") != nullptr;  // phase times on stderr
    auto t0 = std::chrono::steady_clock::now();
    auto lap = [&](const char* what) {
        if (!dbg) return;
        auto t1 = std::chrono::steady_clock::now();
        fprintf(stderr, "[pss] sift.%-10s %8.3f ms\n", what, std::chrono::duration<double, std::milli>(t1 - t0).count());
        t0 = t1;
    };
    std::vector<int64_t> order;
    std::vector<std::pair<int64_t, int64_t>> bk;
    bucket_by_dm(raw, n, P.ndm(), &order, &bk);
    lap("bucket");
    // within each DM trial (independent: in parallel, largest trials first)
    std::vector<std::vector<Item>> surv(bk.size());
    std::vector<int64_t> by_size(bk.size());
    std::iota(by_size.begin(), by_size.end(), 0);
    std::stable_sort(by_size.begin(), by_size.end(), [&](int64_t x, int64_t y) {
        return bk[(size_t)x].second - bk[(size_t)x].first > bk[(size_t)y].second - bk[(size_t)y].first;
    });
    parallel_for((int64_t)bk.size(), 1, [&](int64_t bi) {
        const int64_t b = by_size[(size_t)bi];
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
                items[pick_rep(items, G.members.data() + G.start[g], G.start[g + 1] - G.start[g], false)]);
    });
    for (auto& v : surv) out->insert(out->end(), v.begin(), v.end());
    lap("within");
    if (dbg) fprintf(stderr, "[pss] sift: %lld raw, %zu survive their trial\n", (long long)n, out->size());
    return PSS_OK;
}

namespace {
int64_t fdiv64(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
uint64_t cell_hash(int64_t r, int64_t z) {
    uint64_t h = (uint64_t)r * 0x9E3779B97F4A7C15ull ^ ((uint64_t)z + 0x632BE59BD9B4E019ull) * 0xC2B2AE3D27D4EB4Full;
    return h ^ (h >> 29);
}
}  // namespace

int SiftLinker::find_cell(int64_t cr, int64_t cz) const {
    if (table_.empty()) return -1;
    const size_t mask = table_.size() - 1;
    for (size_t h = cell_hash(cr, cz) & mask;; h = (h + 1) & mask) {
        const int c = table_[h];
        if (c < 0) return -1;
        if (cells_[(size_t)c].cr == cr && cells_[(size_t)c].cz == cz) return c;
    }
}

int SiftLinker::root(int c) const {
    while (par_[(size_t)c] != c) {
        par_[(size_t)c] = par_[(size_t)par_[(size_t)c]];
        c = par_[(size_t)c];
    }
    return c;
}

void SiftLinker::grow() {
    size_t cap = table_.empty() ? 1024 : table_.size() * 2;
    while (cap < 2 * (cells_.size() + 1)) cap *= 2;
    table_.assign(cap, -1);
    for (size_t c = 0; c < cells_.size(); ++c)
        for (size_t h = cell_hash(cells_[c].cr, cells_[c].cz) & (cap - 1);; h = (h + 1) & (cap - 1))
            if (table_[h] < 0) {
                table_[h] = (int)c;
                break;
            }
}

void SiftLinker::add(const std::vector<SiftItem>& items, size_t from) {
    for (size_t i = from; i < items.size(); ++i) {
        const SiftItem& x = items[i];
        const int64_t cr = fdiv64(x.kr, 64), cz = fdiv64(x.kz, 32);
        int c = find_cell(cr, cz);
        if (c < 0) {
            if (2 * (cells_.size() + 1) > table_.size()) grow();
            c = (int)cells_.size();
            cells_.push_back(LCell{cr, cz, x.kr, x.kr, x.kz, x.kz, {}});
            par_.push_back(c);
            const size_t mask = table_.size() - 1;
            for (size_t h = cell_hash(cr, cz) & mask;; h = (h + 1) & mask)
                if (table_[h] < 0) {
                    table_[h] = c;
                    break;
                }
        }
        LCell& C = cells_[(size_t)c];
        C.mem.push_back((int)i);
        C.r_lo = std::min(C.r_lo, x.kr);
        C.r_hi = std::max(C.r_hi, x.kr);
        C.z_lo = std::min(C.z_lo, x.kz);
        C.z_hi = std::max(C.z_hi, x.kz);
        cell_of_.push_back(c);
        // the new item's links to the eight neighbouring cells (its own cell's members link to it)
        for (int dr = -1; dr <= 1; ++dr)
            for (int dz = -1; dz <= 1; ++dz) {
                if (dr == 0 && dz == 0) continue;
                const int b = find_cell(cr + dr, cz + dz);
                if (b < 0 || root(b) == root(c)) continue;
                const LCell& B = cells_[(size_t)b];
                if (B.r_lo - x.kr > 64 || x.kr - B.r_hi > 64 || B.z_lo - x.kz > 32 || x.kz - B.z_hi > 32) continue;
                for (int q : B.mem) {
                    const SiftItem& y = items[(size_t)q];
                    if (std::llabs(x.kr - y.kr) <= 64 && std::llabs(x.kz - y.kz) <= 32) {
                        const int ra = root(c), rb = root(b);
                        par_[(size_t)std::max(ra, rb)] = std::min(ra, rb);
                        break;
                    }
                }
            }
    }
}

void SiftLinker::groups(std::vector<int>* start, std::vector<int>* members) const {
    const int nc = (int)cells_.size();
    std::vector<int> slot((size_t)nc, -1), cnt;
    int ng = 0;
    for (int c = 0; c < nc; ++c) {
        const int r = root(c);
        if (slot[(size_t)r] < 0) {
            slot[(size_t)r] = ng++;
            cnt.push_back(0);
        }
        cnt[(size_t)slot[(size_t)r]] += (int)cells_[(size_t)c].mem.size();
    }
    start->assign((size_t)ng + 1, 0);
    for (int g = 0; g < ng; ++g) (*start)[(size_t)g + 1] = (*start)[(size_t)g] + cnt[(size_t)g];
    members->resize(cell_of_.size());
    std::vector<int> fill(start->begin(), start->end() - 1);
    for (int c = 0; c < nc; ++c) {
        const int g = slot[(size_t)root(c)];
        for (int i : cells_[(size_t)c].mem) (*members)[(size_t)fill[(size_t)g]++] = i;
    }
}

pss_status sift_across(const Plan& P, const pss_search_cfg& cfg, std::vector<SiftItem>& survivors,
                       std::vector<pss_cand>* out, const SiftLinker* linked) {
    out->clear();
    const bool dbg = getenv("PSS_TIMING") != nullptr;
    auto t0 = std::chrono::steady_clock::now();
    auto lap = [&](const char* what) {
        if (!dbg) return;
        auto t1 = std::chrono::steady_clock::now();
        fprintf(stderr, "[pss] sift.%-10s %8.3f ms\n", what, std::chrono::duration<double, std::milli>(t1 - t0).count());
        t0 = t1;
    };
    Groups G;
    if (linked && linked->size() == survivors.size()) linked->groups(&G.start, &G.members);
    else G = link_groups(survivors, cfg.dz);
    lap("link");
    // one representative per group, groups in parallel (each writes its own slot); tasks of
    // about ng / 256 groups: one group per task when they are few (about 100 on the drift-scan
    // file, the largest spanning hundreds of trials), runs of them when they are many (35 k on
    // the accel file, where single-group tasks contend for the task counter)
    const int ng = G.count();
    std::vector<pss_cand> reps((size_t)ng);
    std::vector<char> keep((size_t)ng, 0);
    parallel_for(ng, std::max(1, ng / 256), [&](int64_t g) {
        const int* mem = G.members.data() + G.start[g];
        const int nm = G.start[g + 1] - G.start[g];
        int hits = 1;
        if (nm > 1) {
            // distinct DM trials of the group: a bit per trial, cleared again after the count
            thread_local std::vector<uint64_t> seen;
            const size_t words = (size_t)(P.ndm() + 63) / 64;
            if (seen.size() < words) seen.assign(words, 0);
            hits = 0;
            for (int q = 0; q < nm; ++q) {
                const int32_t d = survivors[mem[q]].dm_idx;
                const uint64_t bit = 1ull << (d & 63);
                if (!(seen[(size_t)(d >> 6)] & bit)) {
                    seen[(size_t)(d >> 6)] |= bit;
                    ++hits;
                }
            }
            for (int q = 0; q < nm; ++q) seen[(size_t)(survivors[mem[q]].dm_idx >> 6)] = 0;
        }
        // groups seen in too few trials are dropped before any sigma is evaluated
        if (hits < cfg.min_dm_hits) return;
        const int best = pick_rep(survivors, mem, nm, true);
        const Item& b = survivors[best];
        pss_cand& c = reps[(size_t)g];
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
        keep[(size_t)g] = 1;
    });
    for (int g = 0; g < ng; ++g)
        if (keep[(size_t)g]) out->push_back(reps[(size_t)g]);
    lap("reps");
    // order by (DM index, numharm, r, z): a counting sort by DM index, then each trial's
    // candidates sorted in parallel
    const int64_t nd = P.ndm();
    std::vector<int64_t> first((size_t)nd + 1, 0);
    for (const pss_cand& c : *out) first[(size_t)c.dm_idx + 1]++;
    for (int64_t d = 0; d < nd; ++d) first[(size_t)d + 1] += first[(size_t)d];
    std::vector<pss_cand> sorted(out->size());
    {
        std::vector<int64_t> pos(first.begin(), first.end() - 1);
        for (const pss_cand& c : *out) sorted[(size_t)pos[(size_t)c.dm_idx]++] = c;
    }
    parallel_for(nd, std::max<int64_t>(1, nd / 256), [&](int64_t d) {
        std::sort(sorted.begin() + first[(size_t)d], sorted.begin() + first[(size_t)d + 1],
                  [](const pss_cand& a, const pss_cand& b) {
                      if (a.numharm != b.numharm) return a.numharm < b.numharm;
                      if (a.r != b.r) return a.r < b.r;
                      return a.z < b.z;
                  });
    });
    out->swap(sorted);
    lap("sort");
    return PSS_OK;
}

pss_status sift(const Plan& P, const pss_search_cfg& cfg, const pss_raw_cand* raw, int64_t n,
                std::vector<pss_cand>* out) {
    std::vector<SiftItem> survivors;
    PSS_TRY(sift_within(P, cfg, raw, n, &survivors));
    return sift_across(P, cfg, survivors, out);
}

}  // namespace pss
