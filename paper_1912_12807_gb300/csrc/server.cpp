// Serving: continuous batching of filterbank files on one device.
//
// The paper processes a drift-scan survey whose files arrive every ~26 s and
// must each be searched within that time (Sect. 1); on CPUs it keeps up by
// running up to a "parallel number" of PRESTO processes at once and starting
// a new one as soon as a slot frees (its V3 scheme, Sect. 2).  Here each of
// max_slots worker threads is a slot that runs one file at a time through a
// prepared, graph-captured search (pss_batch, its own stream).  A queued
// file is admitted in arrival order as soon as a slot is free: it reuses an
// idle prepared batch of its shape (descriptor, plan, search parameters) if
// there is one, otherwise a new batch is prepared when the file's estimated
// device footprint fits in what is left of the budget, evicting least
// recently used idle batches of other shapes to make room.  The kernels of
// the files in flight overlap on the GPU, and each slot sifts its file on
// the host while the others compute.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <sstream>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pss_internal.h"

struct pss_result {
    pss_status status = PSS_OK;
    std::string err;
    std::vector<pss_cand> cands;
    double latency_s = 0.0;
};

namespace pss {
namespace {

using Clock = std::chrono::steady_clock;

// Page-locked host buffers that hold queued files: the copy into one at
// submit is a plain memcpy (split over threads), and the slot's upload from
// it is an asynchronous DMA instead of the driver's staged pageable copy.
// At most `cap` bytes are kept; past that, files wait in ordinary memory.
class PinnedPool {
  public:
    explicit PinnedPool(size_t cap) : cap_(cap) {}
    ~PinnedPool() {
        for (auto& b : free_) cudaFreeHost(b.second);
    }
    // a buffer of at least n bytes, or nullptr (then the caller uses pageable memory)
    void* take(size_t n) {
        {
            std::lock_guard<std::mutex> lk(mu_);
            for (size_t i = 0; i < free_.size(); ++i)
                if (free_[i].first >= n) {
                    void* p = free_[i].second;
                    size_[p] = free_[i].first;
                    free_.erase(free_.begin() + (long)i);
                    return p;
                }
            if (held_ + n > cap_) return nullptr;
            held_ += n;
        }
        void* p = nullptr;
        if (cudaHostAlloc(&p, n, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            std::lock_guard<std::mutex> lk(mu_);
            held_ -= n;
            return nullptr;
        }
        std::lock_guard<std::mutex> lk(mu_);
        size_[p] = n;
        return p;
    }
    void give(void* p) {
        if (!p) return;
        std::lock_guard<std::mutex> lk(mu_);
        free_.emplace_back(size_[p], p);
        size_.erase(p);
    }

  private:
    size_t cap_, held_ = 0;
    std::mutex mu_;
    std::vector<std::pair<size_t, void*>> free_;
    std::unordered_map<void*, size_t> size_;
};

void copy_parallel(uint8_t* dst, const uint8_t* src, size_t n) {
    const size_t chunk = (size_t)8 << 20;
    parallel_for((int64_t)((n + chunk - 1) / chunk), 1, [&](int64_t i) {
        const size_t b = (size_t)i * chunk, e = std::min(n, b + chunk);
        memcpy(dst + b, src + b, e - b);
    });
}

struct Request {
    uint64_t ticket = 0;
    PinnedPool* pool = nullptr;
    void* pinned = nullptr;
    std::vector<uint8_t> data;  // used when no pinned buffer was available
    pss_fil_desc fil{};
    std::vector<uint8_t> mask;
    std::vector<pss_dd_stage> stages;
    pss_search_cfg cfg{};
    pss_plan* plan = nullptr;
    size_t estimate = 0;
    std::string key;
    Clock::time_point t_submit;
    const void* bytes() const { return pinned ? pinned : (const void*)data.data(); }
    void release_data() {
        if (pinned) pool->give(pinned);
        pinned = nullptr;
        std::vector<uint8_t>().swap(data);
    }
    ~Request() {
        release_data();
        if (plan) pss_plan_free(plan);
    }
};

std::string shape_key(const pss_fil_desc& f, const std::vector<uint8_t>& mask, const std::vector<pss_dd_stage>& st,
                      const pss_search_cfg& c, int32_t nsub, int32_t group) {
    std::ostringstream o;
    o << "sub" << nsub << ',' << group << '|';
    o.precision(17);
    o << f.nchan << '/' << f.nbits << '/' << f.nsamp << '/' << f.tsamp_s << '/' << f.fch0_mhz << '/' << f.foff_mhz
      << '/' << f.layout << '|';
    for (uint8_t m : mask) o << (m ? '1' : '0');
    o << '|';
    for (const auto& s : st) o << s.dm_lo << ',' << s.dm_step << ',' << s.n_dm << ',' << s.ds << ';';
    o << '|' << c.zmax << ',' << c.numharm << ',' << c.dz << ',' << c.sigma_thr << ',' << c.f_lo_hz << ','
      << c.whiten_block << ',' << c.halfwidth_extra << ',' << c.min_dm_hits;
    return o.str();
}

// A prepared batch not in use, with the time it was last used.
struct Idle {
    pss_batch* batch;
    std::string key;
    size_t bytes;
    uint64_t stamp;
};

}  // namespace
}  // namespace pss

using namespace pss;

struct pss_server {
    int device = 0;
    size_t budget = 0;
    PinnedPool pinned{(size_t)4 << 30};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<uint64_t, pss_result*> done;
    std::unordered_map<uint64_t, bool> known;  // submitted and not yet handed out
    uint64_t next_ticket = 1;
    size_t in_use = 0;
    bool stop = false;
    std::vector<Idle> idle;  // prepared batches no slot is using (any shape)
    uint64_t clock = 0;
    std::vector<std::thread> workers;
    std::vector<double> latencies;
    // grouped mode (max_group > 1): each slot searches up to max_group queued
    // files at once through pss_search_multi on a context of its own; held[i]
    // is what slot i's context holds on the device
    int max_group = 1;
    std::vector<size_t> held;
    int64_t groups_run = 0, files_grouped = 0;

    void finish(Request* r, pss_result* res) {
        res->latency_s = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
        std::lock_guard<std::mutex> lk(mu);
        done[r->ticket] = res;
        latencies.push_back(res->latency_s);
        cv_done.notify_all();
        cv_work.notify_all();
    }

    // Admission of the file at the head of the queue (FIFO), under `mu`:
    // reuse an idle batch of its shape; else prepare a new one if its
    // estimated footprint fits in what is left of the budget; else free the
    // least recently used idle batch and try again; else wait for a running
    // file to finish.  Returns the request, with *batch set when one was
    // reused (and *reserved = bytes set aside for a new batch otherwise).
    Request* admit(std::unique_lock<std::mutex>& lk, pss_batch** batch, size_t* reserved) {
        while (!stop) {
            if (queue.empty()) {
                cv_work.wait(lk);
                continue;
            }
            Request* h = queue.front();
            if (h->estimate > budget) {
                queue.pop_front();
                lk.unlock();
                pss_result* res = new pss_result();
                res->status = PSS_ENOMEM;
                res->err = "file needs more device memory than the server budget";
                finish(h, res);
                delete h;
                lk.lock();
                continue;
            }
            for (size_t i = 0; i < idle.size(); ++i)
                if (idle[i].key == h->key) {
                    *batch = idle[i].batch;
                    *reserved = 0;
                    idle.erase(idle.begin() + (long)i);
                    queue.pop_front();
                    return h;
                }
            if (in_use + h->estimate <= budget) {
                in_use += h->estimate;
                *batch = nullptr;
                *reserved = h->estimate;
                queue.pop_front();
                return h;
            }
            if (!idle.empty()) {
                size_t lru = 0;
                for (size_t i = 1; i < idle.size(); ++i)
                    if (idle[i].stamp < idle[lru].stamp) lru = i;
                Idle v = idle[lru];
                idle.erase(idle.begin() + (long)lru);
                in_use -= v.bytes;
                lk.unlock();
                pss_batch_free(v.batch);
                lk.lock();
                continue;
            }
            cv_work.wait(lk);
        }
        return nullptr;
    }

    // Whether r can join a group led by h: an exact plan and the same search parameters.
    static bool groupable(const Request* h, const Request* r) {
        const pss_search_cfg &a = h->cfg, &b = r->cfg;
        return r->plan->nsub == 0 && h->plan->nsub == 0 && a.zmax == b.zmax && a.numharm == b.numharm &&
               a.dz == b.dz && a.sigma_thr == b.sigma_thr && a.f_lo_hz == b.f_lo_hz &&
               a.whiten_block == b.whiten_block && a.halfwidth_extra == b.halfwidth_extra &&
               a.min_dm_hits == b.min_dm_hits;
    }
    static size_t group_bytes(const std::vector<Request*>& g) {
        std::vector<const Plan*> plans;
        std::vector<const pss_fil_desc*> fils;
        for (const Request* r : g) {
            plans.push_back(r->plan);
            fils.push_back(&r->fil);
        }
        return multi_footprint(plans, fils, &g[0]->cfg);
    }

    // Grouped admission (under `mu`): the head of the queue and the files
    // queued right behind it that can join it, up to max_group, while the
    // group's footprint beyond what this slot's context already holds fits in
    // what is left of the budget.  A file that cannot be grouped (a two-stage
    // plan) runs alone.  A file whose own footprint exceeds the budget fails
    // with PSS_ENOMEM.
    bool admit_group(std::unique_lock<std::mutex>& lk, int wi, std::vector<Request*>* grp, size_t* reserved) {
        while (!stop) {
            if (queue.empty()) {
                cv_work.wait(lk);
                continue;
            }
            Request* h = queue.front();
            if (h->estimate > budget) {
                queue.pop_front();
                lk.unlock();
                pss_result* res = new pss_result();
                res->status = PSS_ENOMEM;
                res->err = "file needs more device memory than the server budget";
                finish(h, res);
                delete h;
                lk.lock();
                continue;
            }
            grp->assign(1, h);
            size_t fp = h->plan->nsub == 0 ? group_bytes(*grp) : h->estimate;
            if (h->plan->nsub == 0) {
                for (size_t i = 1; i < queue.size() && (int)grp->size() < max_group; ++i) {
                    Request* r = queue[i];
                    if (!groupable(h, r)) break;  // arrival order is kept
                    grp->push_back(r);
                    const size_t f2 = group_bytes(*grp);
                    const size_t need2 = f2 > held[wi] ? f2 - held[wi] : 0;
                    if (in_use + need2 > budget) {
                        grp->pop_back();
                        break;
                    }
                    fp = f2;
                }
            }
            const size_t need = fp > held[wi] ? fp - held[wi] : 0;
            if (in_use + need <= budget) {
                for (size_t i = 0; i < grp->size(); ++i) queue.pop_front();
                in_use += need;
                *reserved = need;
                return true;
            }
            cv_work.wait(lk);
        }
        return false;
    }

    void worker_grouped(int wi) {
        cudaSetDevice(device);
        pss_ctx* ctx = nullptr;
        const pss_status cst = pss_ctx_create(device, &ctx);
        const std::string cerr = cst == PSS_OK ? "" : pss_last_error();
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            std::vector<Request*> grp;
            size_t reserved = 0;
            if (!admit_group(lk, wi, &grp, &reserved)) break;  // stopping
            lk.unlock();
            std::vector<pss_result*> res(grp.size());
            for (auto& r : res) r = new pss_result();
            try {
                pss_status st = cst;
                std::string err = cerr;
                std::vector<pss_cand> out;
                std::vector<int64_t> counts(grp.size(), 0);
                if (st == PSS_OK && grp[0]->plan->nsub > 0) {
                    // a two-stage plan runs alone through the single-file path
                    int64_t n = 0;
                    out.resize(1024);
                    st = pss_search_dm_batch(ctx, grp[0]->plan, &grp[0]->fil, grp[0]->bytes(), 0, &grp[0]->cfg, 0,
                                             grp[0]->plan->ndm(), out.data(), (int64_t)out.size(), &n, nullptr);
                    if (st == PSS_ECAP) {
                        out.resize((size_t)n);
                        st = pss_ctx_take_cands(ctx, out.data(), n, &n);
                    }
                    out.resize(st == PSS_OK ? (size_t)n : 0);
                    counts[0] = (int64_t)out.size();
                } else if (st == PSS_OK) {
                    std::vector<pss_multi_file> mf(grp.size());
                    for (size_t i = 0; i < grp.size(); ++i) mf[i] = {grp[i]->plan, &grp[i]->fil, grp[i]->bytes()};
                    int64_t n = 0;
                    out.resize(4096);
                    st = pss_search_multi(ctx, &grp[0]->cfg, mf.data(), (int32_t)grp.size(), 0, out.data(),
                                          (int64_t)out.size(), counts.data(), &n, nullptr);
                    if (st == PSS_ECAP) {
                        out.resize((size_t)n);
                        st = pss_ctx_take_cands(ctx, out.data(), n, &n);
                    }
                    out.resize(st == PSS_OK ? (size_t)n : 0);
                }
                if (st != PSS_OK && err.empty()) err = pss_last_error();
                size_t off = 0;
                for (size_t i = 0; i < grp.size(); ++i) {
                    res[i]->status = st;
                    res[i]->err = err;
                    if (st == PSS_OK) {
                        res[i]->cands.assign(out.begin() + (long)off, out.begin() + (long)(off + counts[i]));
                        off += (size_t)counts[i];
                    }
                }
            } catch (const std::bad_alloc&) {
                for (auto& r : res) {
                    r->status = PSS_ENOMEM;
                    r->err = "host allocation failed";
                }
            }
            {
                const size_t now = ctx ? ctx_device_bytes(ctx) : 0;
                std::lock_guard<std::mutex> g(mu);
                in_use = in_use - reserved - held[wi] + now;
                held[wi] = now;
                ++groups_run;
                files_grouped += (int64_t)grp.size();
            }
            for (size_t i = 0; i < grp.size(); ++i) {
                grp[i]->release_data();
                finish(grp[i], res[i]);
                delete grp[i];
            }
            lk.lock();
        }
        lk.unlock();
        if (ctx) pss_ctx_destroy(ctx);
    }

    void worker(int) {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            pss_batch* batch = nullptr;
            size_t held = 0;
            Request* r = admit(lk, &batch, &held);
            if (!r) return;  // stopping
            if (batch) held = pss_batch_footprint(batch);
            lk.unlock();
            pss_result* res = new pss_result();
            try {
                if (!batch) {
                    pss_status st = pss_batch_create(device, r->plan, &r->fil, &r->cfg, &batch);
                    if (st != PSS_OK) {
                        batch = nullptr;
                        res->status = st;
                        res->err = pss_last_error();
                    } else {
                        const size_t actual = pss_batch_footprint(batch);
                        std::lock_guard<std::mutex> g(mu);
                        in_use = in_use - held + actual;
                        held = actual;
                    }
                }
                if (res->status == PSS_OK) {
                    int64_t n = 0;
                    std::vector<pss_cand> buf(1024);
                    pss_status st = pss_batch_run(batch, r->bytes(), 0, buf.data(), (int64_t)buf.size(), &n, nullptr);
                    if (st == PSS_ECAP) {
                        buf.resize((size_t)n);
                        st = pss_batch_take_cands(batch, buf.data(), (int64_t)buf.size(), &n);
                    }
                    if (st != PSS_OK) {
                        res->status = st;
                        res->err = pss_last_error();
                    } else {
                        buf.resize((size_t)n);
                        res->cands.swap(buf);
                    }
                }
            } catch (const std::bad_alloc&) {
                res->status = PSS_ENOMEM;
                res->err = "host allocation failed";
            }
            // the run's footprint may have grown (a candidate buffer resized on overflow)
            if (batch && res->status == PSS_OK) {
                const size_t actual = pss_batch_footprint(batch);
                std::lock_guard<std::mutex> g(mu);
                in_use = in_use - held + actual;
                held = actual;
                idle.push_back(Idle{batch, r->key, held, ++clock});
            } else {
                // a failed batch is not reused
                if (batch) pss_batch_free(batch);
                std::lock_guard<std::mutex> g(mu);
                in_use -= held;
            }
            r->release_data();
            finish(r, res);
            delete r;
            lk.lock();
        }
    }
};

extern "C" pss_status pss_server_create_grouped(int device, size_t hbm_budget_bytes, int max_slots, int max_group,
                                               pss_server** out) {
    if (!out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0 || max_group < 1 || max_group > 1024)
        return fail(PSS_EINVAL, "pss_server_create: bad arguments");
    *out = nullptr;
    int n = 0;
    PSS_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(PSS_EINVAL, "pss_server_create: no such device");
    pss_server* s = new pss_server();
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->max_group = max_group;
    s->held.assign((size_t)max_slots, 0);
    for (int i = 0; i < max_slots; ++i) {
        if (max_group > 1) s->workers.emplace_back([s, i] { s->worker_grouped(i); });
        else s->workers.emplace_back([s, i] { s->worker(i); });
    }
    *out = s;
    return PSS_OK;
}

extern "C" pss_status pss_server_create(int device, size_t hbm_budget_bytes, int max_slots, pss_server** out) {
    return pss_server_create_grouped(device, hbm_budget_bytes, max_slots, 1, out);
}

// nsub == 0: an exact plan; otherwise a two-stage plan (pss_dd_plan_subband)
static pss_status submit(pss_server* srv, const pss_fil_desc* fil, const void* host_data, const pss_dd_stage* stages,
                         int nstages, int32_t nsub, int32_t group, const pss_search_cfg* cfg, uint64_t* ticket) {
    if (!srv || !fil || !host_data || !stages || nstages <= 0 || !cfg || !ticket)
        return fail(PSS_EINVAL, "pss_submit_file: null argument");
    Request* r = new Request();
    r->fil = *fil;
    if (fil->chan_mask) {
        r->mask.assign(fil->chan_mask, fil->chan_mask + fil->nchan);
        r->fil.chan_mask = r->mask.data();
    }
    r->stages.assign(stages, stages + nstages);
    r->cfg = *cfg;
    pss_status st = nsub > 0 ? pss_dd_plan_subband(&r->fil, r->stages.data(), nstages, nsub, group, &r->plan)
                             : pss_dd_plan(&r->fil, r->stages.data(), nstages, &r->plan);
    if (st != PSS_OK) {
        delete r;
        return st;
    }
    st = validate_search(r->plan, &r->fil, &r->cfg);
    if (st != PSS_OK) {
        delete r;
        return st;
    }
    r->estimate = search_footprint(*r->plan, &r->fil, &r->cfg, kBatchInitialCap);
    const size_t nbytes = fil->nbits == 8 ? (size_t)fil->nchan * fil->nsamp : (size_t)(fil->nchan / 8) * fil->nsamp;
    cudaSetDevice(srv->device);
    r->pool = &srv->pinned;
    r->pinned = srv->pinned.take(nbytes);
    try {
        if (r->pinned) {
            copy_parallel((uint8_t*)r->pinned, (const uint8_t*)host_data, nbytes);
        } else {
            r->data.resize(nbytes);
            copy_parallel(r->data.data(), (const uint8_t*)host_data, nbytes);
        }
    } catch (const std::bad_alloc&) {
        delete r;
        return fail(PSS_ENOMEM, "pss_submit_file: cannot copy the file");
    }
    r->key = shape_key(r->fil, r->mask, r->stages, r->cfg, nsub, group);
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> lk(srv->mu);
    r->ticket = srv->next_ticket++;
    *ticket = r->ticket;
    srv->known[r->ticket] = true;
    srv->queue.push_back(r);
    srv->cv_work.notify_all();
    return PSS_OK;
}

extern "C" pss_status pss_submit_file(pss_server* srv, const pss_fil_desc* fil, const void* host_data,
                                      const pss_dd_stage* stages, int nstages, const pss_search_cfg* cfg,
                                      uint64_t* ticket) {
    return submit(srv, fil, host_data, stages, nstages, 0, 0, cfg, ticket);
}

extern "C" pss_status pss_submit_file_subband(pss_server* srv, const pss_fil_desc* fil, const void* host_data,
                                              const pss_dd_stage* stages, int nstages, int32_t nsub, int32_t group,
                                              const pss_search_cfg* cfg, uint64_t* ticket) {
    if (nsub <= 0) return fail(PSS_EINVAL, "pss_submit_file_subband: nsub must be > 0");
    return submit(srv, fil, host_data, stages, nstages, nsub, group, cfg, ticket);
}

extern "C" pss_status pss_poll(pss_server* srv, uint64_t ticket, int timeout_ms, pss_result** out) {
    if (!srv || !out) return fail(PSS_EINVAL, "pss_poll: null argument");
    *out = nullptr;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (!srv->known.count(ticket)) return fail(PSS_EINVAL, "pss_poll: unknown ticket (or already handed out)");
    auto ready = [&] { return srv->done.count(ticket) > 0; };
    if (!ready()) {
        if (timeout_ms == 0) return fail(PSS_ENOTREADY, "pss_poll: not ready");
        if (timeout_ms < 0) srv->cv_done.wait(lk, ready);
        else if (!srv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
            return fail(PSS_ETIMEOUT, "pss_poll: wait expired");
    }
    *out = srv->done[ticket];
    srv->done.erase(ticket);
    srv->known.erase(ticket);
    return PSS_OK;
}

extern "C" pss_status pss_result_cands(const pss_result* r, const pss_cand** c, int64_t* n, double* latency_s) {
    if (!r) return fail(PSS_EINVAL, "pss_result_cands: null result");
    if (c) *c = r->cands.empty() ? nullptr : r->cands.data();
    if (n) *n = (int64_t)r->cands.size();
    if (latency_s) *latency_s = r->latency_s;
    if (r->status != PSS_OK) set_error(r->err);
    return r->status;
}

extern "C" void pss_result_free(pss_result* r) { delete r; }

extern "C" pss_status pss_server_stats(pss_server* srv, int64_t* completed, double* p50_s, double* p99_s,
                                       size_t* bytes_in_use) {
    if (!srv) return fail(PSS_EINVAL, "pss_server_stats: null server");
    std::lock_guard<std::mutex> lk(srv->mu);
    std::vector<double> v = srv->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) {
        if (v.empty()) return 0.0;
        // nearest-rank percentile
        size_t i = (size_t)ceil(p / 100.0 * (double)v.size());
        if (i < 1) i = 1;
        return v[i - 1];
    };
    if (completed) *completed = (int64_t)v.size();
    if (p50_s) *p50_s = pct(50.0);
    if (p99_s) *p99_s = pct(99.0);
    if (bytes_in_use) *bytes_in_use = srv->in_use;
    return PSS_OK;
}

extern "C" pss_status pss_server_group_stats(pss_server* srv, int64_t* groups, int64_t* files) {
    if (!srv) return fail(PSS_EINVAL, "pss_server_group_stats: null server");
    std::lock_guard<std::mutex> lk(srv->mu);
    if (groups) *groups = srv->groups_run;
    if (files) *files = srv->files_grouped;
    return PSS_OK;
}

extern "C" void pss_server_destroy(pss_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    for (auto& t : srv->workers) t.join();
    for (auto& v : srv->idle) pss_batch_free(v.batch);
    for (Request* r : srv->queue) delete r;
    for (auto& kv : srv->done) delete kv.second;
    delete srv;
}
