// C-ABI entry points of libpss: context, plan, and the search path
// dedisperse -> FFT -> whiten -> f-fdot plane -> harmonic sum -> sift
// (paper Sect. 2, steps 2-5).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pss_internal.h"
#include "response.cuh"

namespace pss {

// pss_debug_fail_alloc: device allocations left before one is made to fail (<= 0: none)
std::atomic<int64_t> g_alloc_countdown{0};

pss_status DevBuf::ensure(size_t want) {
    if (want <= bytes) return PSS_OK;
    release();
    size_t sz = want + want / 8 + 256;
    if (g_alloc_countdown.load() > 0 && g_alloc_countdown.fetch_sub(1) == 1)
        return fail(PSS_ENOMEM, "device allocation of " + std::to_string(sz) + " bytes refused (pss_debug_fail_alloc)");
    cudaError_t e = cudaMalloc(&p, sz);
    if (e != cudaSuccess) {
        p = nullptr;
        bytes = 0;
        cudaGetLastError();
        return fail(PSS_ENOMEM, std::string("device allocation of ") + std::to_string(sz) + " bytes failed: " +
                                    cudaGetErrorString(e));
    }
    bytes = sz;
    return PSS_OK;
}

void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

ProfScope::ProfScope(Ctx* ctx, int st, cudaStream_t str) : c(ctx), stage(st), s(str) {
    if (!c->prof_on) return;
    for (int i = 0; i < 2; ++i) {
        cudaEvent_t e = nullptr;
        if (!c->prof_pool.empty()) {
            e = c->prof_pool.back();
            c->prof_pool.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
        }
        (i == 0 ? a : b) = e;
    }
    if (a) cudaEventRecord(a, s);
}

ProfScope::~ProfScope() {
    if (!a || !b) return;
    cudaEventRecord(b, s);
    c->prof_recs.push_back({stage, a, b});
}

namespace {

// Host phase timing, printed to stderr when PSS_TIMING is set in the
// environment (tracing of the host side of a call).
struct HostTimer {
    bool on;
    std::chrono::steady_clock::time_point t;
    HostTimer() : on(getenv("PSS_TIMING") != nullptr), t(std::chrono::steady_clock::now()) {}
    void mark(const char* what) {
        if (!on) return;
        auto n = std::chrono::steady_clock::now();
        fprintf(stderr, "[pss] %-14s %8.3f ms\n", what, std::chrono::duration<double>(n - t).count() * 1e3);
        t = n;
    }
};

// NULL selects the legacy default stream (stream handle 0 in a library
// compiled without per-thread default streams).
cudaStream_t pick_stream(pss_ctx* ctx, void* stream) {
    (void)ctx;
    return (cudaStream_t)stream;
}

pss_status check_common(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data,
                        int64_t dm_begin, int64_t dm_end) {
    if (!ctx || !plan || !fil || !data) return fail(PSS_EINVAL, "null ctx, plan, descriptor or data");
    if (fil->nchan != plan->nchan || fil->nsamp != plan->nsamp)
        return fail(PSS_EINVAL, "descriptor does not match the plan (nchan/nsamp)");
    if (fil->nbits != 8 && fil->nbits != 1) return fail(PSS_EINVAL, "nbits must be 8 or 1");
    if (fil->nbits == 1 && (fil->nchan % 8) != 0) return fail(PSS_EINVAL, "1-bit data needs nchan % 8 == 0");
    if (fil->layout != 0 && fil->layout != 1) return fail(PSS_EINVAL, "layout must be 0 or 1");
    if (fil->layout == 1 && fil->nbits != 8) return fail(PSS_EINVAL, "channel-major layout is 8-bit only");
    if (dm_begin < 0 || dm_end > plan->ndm() || dm_begin > dm_end)
        return fail(PSS_EINVAL, "DM range outside the plan");
    return PSS_OK;
}

int64_t file_bytes(const pss_fil_desc* fil) {
    if (fil->nbits == 8) return (int64_t)fil->nchan * fil->nsamp;
    return (int64_t)(fil->nchan / 8) * fil->nsamp;
}

// Row pitch of the channel-major copy: the samples, one tile and the copy
// slack past the end; for a two-stage plan also the furthest stage 1 can
// read past the file (its rows run to N_v ds + the batch's largest D_b for
// every subband; what it reads there never reaches an output).
int64_t xcm_pitch(const Plan& plan, const pss_fil_desc* fil) {
    int64_t extra = 0;
    if (plan.nsub > 0) {
        const int C = plan.nchan, nsub = plan.nsub;
        for (int64_t i = 0; i < plan.ndm(); ++i) {
            int32_t emax = 0, dmax = 0;
            const int32_t* e = &plan.sub_e[(size_t)plan.grp_of[i] * C];
            for (int c = 0; c < C; ++c) emax = std::max(emax, e[c]);
            for (int b = 0; b < nsub; ++b) dmax = std::max(dmax, plan.sub_D[(size_t)i * nsub + b]);
            extra = std::max<int64_t>(extra, (int64_t)emax + dmax - plan.max_delay);
        }
    }
    return ((fil->nsamp + dedisp_tile_samples() + 256 + extra) + 63) / 64 * 64;
}

std::vector<int32_t> kept_channels(const pss_fil_desc* fil) {
    std::vector<int32_t> keep;
    for (int c = 0; c < fil->nchan; ++c)
        if (!fil->chan_mask || fil->chan_mask[c]) keep.push_back(c);
    return keep;
}

// delays of the kept channels, [dm_end - dm_begin][keep.size()]
std::vector<int32_t> compact_delays(const pss_plan* plan, const std::vector<int32_t>& keep, int64_t dm_begin,
                                    int64_t dm_end) {
    const size_t ck = keep.size();
    std::vector<int32_t> hd((size_t)(dm_end - dm_begin) * ck);
    for (int64_t i = 0; i < dm_end - dm_begin; ++i)
        for (size_t r = 0; r < ck; ++r)
            hd[(size_t)i * ck + r] = plan->delays[(size_t)(dm_begin + i) * plan->nchan + keep[r]];
    return hd;
}

// Tables of the two-stage scheme for [dm_begin, dm_end), appended to the
// keep list in ctx->delays_dev (offsets in int32 elements from its start):
//   E   [groups][ck]   within-subband delays of the kept channels,
//   D   [trials][nsub] subband delays,
//   grp [groups]       (first trial - dm_begin, count),
//   z   [nsub]         (first kept channel, kept channels) of each subband.
struct SubTab {
    bool on = false;
    int64_t g_begin = 0;  // first group whose rows are uploaded
    int64_t e_off = 0, d_off = 0, grp_off = 0, z_off = 0;
    int32_t ckmax = 0;    // most kept channels in one subband
    std::vector<int32_t> e_host;  // E as uploaded (host copy for launch sizing)
};

void subband_tables(const pss_plan* plan, const std::vector<int32_t>& keep, int64_t dm_begin, int64_t dm_end,
                    std::vector<int32_t>* host, SubTab* T) {
    const int32_t ck = (int32_t)keep.size();
    const int nsub = plan->nsub, S = plan->sub_S, C = plan->nchan;
    T->on = true;
    T->g_begin = dm_end > dm_begin ? plan->grp_of[dm_begin] : 0;
    const int64_t g_end = dm_end > dm_begin ? plan->grp_of[dm_end - 1] + 1 : T->g_begin;
    const int64_t ng = g_end - T->g_begin, nt = dm_end - dm_begin;
    // int2 tables (grp, z) start on 8-byte boundaries: every offset is kept a multiple of 4 elements
    auto up4 = [](int64_t v) { return (v + 3) & ~int64_t(3); };
    T->e_off = up4(ck);
    T->d_off = up4(T->e_off + ng * ck);
    T->grp_off = up4(T->d_off + nt * nsub);
    T->z_off = up4(T->grp_off + 2 * ng);
    host->assign((size_t)(T->z_off + 2 * nsub), 0);
    int32_t* h = host->data();
    for (int32_t r = 0; r < ck; ++r) h[r] = keep[r];
    for (int64_t g = 0; g < ng; ++g)
        for (int32_t r = 0; r < ck; ++r) h[T->e_off + g * ck + r] = plan->sub_e[(size_t)(T->g_begin + g) * C + keep[r]];
    for (int64_t i = 0; i < nt; ++i)
        for (int b = 0; b < nsub; ++b) h[T->d_off + i * nsub + b] = plan->sub_D[(size_t)(dm_begin + i) * nsub + b];
    for (int64_t g = 0; g < ng; ++g) {
        h[T->grp_off + 2 * g] = (int32_t)(plan->grp_first[T->g_begin + g] - dm_begin);
        h[T->grp_off + 2 * g + 1] = plan->grp_n[T->g_begin + g];
    }
    T->ckmax = 0;
    int32_t r = 0;
    for (int b = 0; b < nsub; ++b) {
        const int32_t first = r;
        while (r < ck && keep[r] < (b + 1) * S) ++r;
        h[T->z_off + 2 * b] = first;
        h[T->z_off + 2 * b + 1] = r - first;
        T->ckmax = std::max(T->ckmax, r - first);
    }
    T->e_host.assign(h + T->e_off, h + T->e_off + ng * ck);
}

// Host-side set-up for a file: the kept channels, their delays for
// [dm_begin, dm_end) (or the two-stage tables, `T`) uploaded to
// ctx->delays_dev, and the channel-major buffer.  Synchronises `s` (the
// delay upload reads a host vector).
pss_status setup_input(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, int64_t dm_begin,
                       int64_t dm_end, cudaStream_t s, int32_t* ck_out, int64_t* pitch_out, SubTab* T = nullptr) {
    const std::vector<int32_t> keep = kept_channels(fil);
    const int32_t ck = (int32_t)keep.size();
    if (ck == 0) return fail(PSS_EINVAL, "channel mask removes every channel");
    const int64_t pitch = xcm_pitch(*plan, fil);
    std::vector<int32_t> host;
    if (plan->nsub > 0) {
        if (!T) return fail(PSS_EINVAL, "internal: two-stage plan without its tables");
        subband_tables(plan, keep, dm_begin, dm_end, &host, T);
    } else {
        // keep list + compacted delays in one upload
        const std::vector<int32_t> hd = compact_delays(plan, keep, dm_begin, dm_end);
        host.resize((size_t)ck + hd.size());
        memcpy(host.data(), keep.data(), sizeof(int32_t) * ck);
        if (!hd.empty()) memcpy(host.data() + ck, hd.data(), sizeof(int32_t) * hd.size());
        if (T) T->on = false;
    }
    // the same tables as the last call (same plan, mask and trials) need no upload and no wait
    const void* before = ctx->delays_dev.p;
    PSS_TRY(ctx->delays_dev.ensure(host.size() * sizeof(int32_t)));
    const bool same = ctx->delays_dev.p == before && ctx->delays_host == host;
    if (!same) {
        ctx->delays_host.clear();
        PSS_CUDA(cudaMemcpyAsync(ctx->delays_dev.p, host.data(), host.size() * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, s));
    }
    PSS_TRY(ctx->xcm.ensure((size_t)ck * pitch + 64));
    // the boxcar table of the downsampled rows (exact plans only)
    if (plan->nsub == 0) {
        size_t need_bx = 0;
        for (const auto& st : plan->stages)
            if (st.n_dm > 0 && st.first < dm_end && st.first + st.n_dm > dm_begin && bx_use(ctx->tune, st.ds) &&
                ck <= 65535)
                need_bx = std::max(need_bx, bx_table_bytes(ck, plan->nsamp, st.ds));
        if (need_bx) {
            const void* was = ctx->bx.p;
            PSS_TRY(ctx->bx.ensure(need_bx));
            if (ctx->bx.p != was) ctx->bx_ds = 0;
        }
    }
    if (!ctx->errflag.p) {
        PSS_TRY(ctx->errflag.ensure(sizeof(int)));
        PSS_CUDA(cudaMemsetAsync(ctx->errflag.p, 0, sizeof(int), s));
    }
    if (!same) {
        PSS_CUDA(cudaStreamSynchronize(s));  // `host` is about to go out of scope
        ctx->delays_host.swap(host);
        ctx->delays_gen++;
    }
    *ck_out = ck;
    *pitch_out = pitch;
    return PSS_OK;
}

// Upload a host file into ctx->fil_dev (device data is used in place).
pss_status upload_input(pss_ctx* ctx, const pss_fil_desc* fil, const void* data, int on_device, cudaStream_t s,
                        const uint8_t** src) {
    *src = (const uint8_t*)data;
    if (on_device) return PSS_OK;
    const int64_t nbytes = file_bytes(fil);
    PSS_TRY(ctx->fil_dev.ensure((size_t)nbytes));
    PSS_CUDA(cudaMemcpyAsync(ctx->fil_dev.p, data, (size_t)nbytes, cudaMemcpyHostToDevice, s));
    *src = (const uint8_t*)ctx->fil_dev.p;
    return PSS_OK;
}

// Unpack/transpose the file into ctx->xcm (kernel launch only).
pss_status enqueue_prep(pss_ctx* ctx, const pss_fil_desc* fil, const uint8_t* src, int32_t ck, int64_t pitch,
                        cudaStream_t s) {
    PrepArgs pa;
    pa.src = src;
    pa.nchan = fil->nchan;
    pa.nbits = fil->nbits;
    pa.layout = fil->layout;
    pa.nsamp = fil->nsamp;
    pa.keep = (const int32_t*)ctx->delays_dev.p;
    pa.ck = ck;
    pa.xcm = (uint8_t*)ctx->xcm.p;
    pa.pitch = pitch;
    ProfScope ps(ctx, 0, s);
    PSS_CUDA(launch_prep(pa, s));
    ctx->bx_ds = 0;  // the boxcar table no longer matches the channel-major data
    return PSS_OK;
}

// Old entry used by pss_dedisperse: set-up, upload and unpack in one go.
pss_status stage_input(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data,
                       int on_device, int64_t dm_begin, int64_t dm_end, cudaStream_t s, int32_t* ck_out,
                       int64_t* pitch_out, SubTab* T) {
    PSS_TRY(setup_input(ctx, plan, fil, dm_begin, dm_end, s, ck_out, pitch_out, T));
    const uint8_t* src = nullptr;
    PSS_TRY(upload_input(ctx, fil, data, on_device, s, &src));
    return enqueue_prep(ctx, fil, src, *ck_out, *pitch_out, s);
}

// max over the dedispersion kernel's groups of consecutive trials and over
// channels of (dmax - dmin)
int32_t delay_spread(const int32_t* d, int64_t nb, int32_t ck) {
    const int G = dedisp_group_trials();
    int32_t sp = 0;
    for (int64_t g = 0; g < nb; g += G) {
        const int64_t ge = std::min<int64_t>(nb, g + G);
        for (int32_t c = 0; c < ck; ++c) {
            int32_t lo = d[g * ck + c], hi = lo;
            for (int64_t i = g + 1; i < ge; ++i) {
                lo = std::min(lo, d[i * ck + c]);
                hi = std::max(hi, d[i * ck + c]);
            }
            sp = std::max(sp, hi - lo);
        }
    }
    return sp;
}

// Launch sizes of one two-stage batch: trials [b0, b0 + nb) of a stage.
struct SubBatch {
    int64_t g_lo = 0;     // first group touched (global index)
    int32_t ngb = 0;      // groups touched
    int64_t len1 = 0;     // stage-1 samples per row: N_v ds + the batch's largest D
    int64_t stride1 = 0;  // row stride of the stage-1 buffer
    int32_t spread1 = 0;  // stage 1: within-subband delay spread over rows of 16 groups
    int32_t spread2 = 0;  // stage 2: subband delay spread within a group
};

SubBatch sub_batch(const pss_plan* plan, const SubTab& T, int32_t ck, int64_t dm_begin, int64_t b0, int32_t nb,
                   int64_t nv, int32_t ds) {
    SubBatch B;
    const int nsub = plan->nsub;
    B.g_lo = plan->grp_of[b0];
    B.ngb = (int32_t)(plan->grp_of[b0 + nb - 1] - B.g_lo + 1);
    int32_t dmax = 0;
    for (int64_t i = b0; i < b0 + nb; ++i)
        for (int b = 0; b < nsub; ++b) dmax = std::max(dmax, plan->sub_D[(size_t)i * nsub + b]);
    B.len1 = nv * ds + dmax;
    B.stride1 = (B.len1 + 3) & ~int64_t(3);
    const int G = dedisp_group_trials();
    const int32_t* e = T.e_host.data() + (B.g_lo - T.g_begin) * ck;
    for (int32_t g = 0; g < B.ngb; g += G) {
        const int32_t ge = std::min<int32_t>(B.ngb, g + G);
        for (int32_t c = 0; c < ck; ++c) {
            int32_t lo = e[(int64_t)g * ck + c], hi = lo;
            for (int32_t k = g + 1; k < ge; ++k) {
                lo = std::min(lo, e[(int64_t)k * ck + c]);
                hi = std::max(hi, e[(int64_t)k * ck + c]);
            }
            B.spread1 = std::max(B.spread1, hi - lo);
        }
    }
    for (int64_t g = B.g_lo; g < B.g_lo + B.ngb; ++g) {
        const int64_t lo = std::max<int64_t>(b0, plan->grp_first[g]);
        const int64_t hi = std::min<int64_t>(b0 + nb, plan->grp_first[g] + plan->grp_n[g]);
        for (int b = 0; b < nsub; ++b) {
            int32_t mn = INT32_MAX, mx = INT32_MIN;
            for (int64_t i = lo; i < hi; ++i) {
                mn = std::min(mn, plan->sub_D[(size_t)i * nsub + b]);
                mx = std::max(mx, plan->sub_D[(size_t)i * nsub + b]);
            }
            if (hi > lo) B.spread2 = std::max(B.spread2, mx - mn);
        }
    }
    (void)dm_begin;
    return B;
}

// Dedisperse trials [b0, b0 + nb) of one stage into rows of out_stride
// (float out_f with per-trial sums, or int32 out_i): the exact kernel, or,
// for a two-stage plan, stage 1 into `subu` and stage 2 from it.  `spread`
// is the exact kernel's delay spread; `SB` the two-stage launch sizes.
pss_status enqueue_dedisp(pss_ctx* ctx, const pss_plan* plan, int32_t ck, int64_t pitch, const SubTab& T,
                          const StageInfo& st, int64_t dm_begin, int64_t b0, int32_t nb, int32_t spread,
                          const SubBatch& SB, void* subu, float* out_f, int32_t* out_i, int64_t out_stride,
                          unsigned long long* sums, cudaStream_t s) {
    const int32_t* base = (const int32_t*)ctx->delays_dev.p;
    // downsampled row: one boxcar table per ds (built once per file and ds), then one term per channel;
    // a few trials alone do not pay for building the table
    if (!T.on && bx_use(ctx->tune, st.ds) && ck <= 65535 && ctx->bx.bytes >= bx_table_bytes(ck, plan->nsamp, st.ds) &&
        (ctx->bx_ds == st.ds || nb >= 16)) {
        if (ctx->bx_ds != st.ds) {
            ProfScope pt(ctx, 6, s);
            BxTableArgs ta{};
            ta.xcm = (const uint8_t*)ctx->xcm.p;
            ta.pitch = pitch;
            ta.ck = ck;
            ta.nsamp = plan->nsamp;
            ta.lds = ilog2(st.ds);
            ta.lmt = ilog2(bx_table_cols(st.ds));
            ta.mlen = bx_mlen(plan->nsamp, st.ds);
            ta.mstride = bx_mstride(plan->nsamp, st.ds);
            ta.table = (uint16_t*)ctx->bx.p;
            PSS_CUDA(launch_bx_table(ta, s));
            ctx->bx_ds = st.ds;
        }
        ProfScope ps(ctx, 1, s);
        BxArgs ba{};
        ba.table = (const uint16_t*)ctx->bx.p;
        ba.mstride = bx_mstride(plan->nsamp, st.ds);
        ba.ck = ck;
        ba.lds = ilog2(st.ds);
        ba.delays = base + ck + (b0 - dm_begin) * ck;
        ba.nb = nb;
        ba.nv = st.nv;
        ba.out_f = out_f;
        ba.out_i = out_i;
        ba.out_stride = out_stride;
        ba.sums = sums;
        PSS_CUDA(launch_dedisp_bx(ba, s));
        return PSS_OK;
    }
    if (!T.on) {
        DedispArgs da{};
        da.xcm = (const uint8_t*)ctx->xcm.p;
        da.pitch = pitch;
        da.ck = ck;
        da.delays = base + ck + (b0 - dm_begin) * ck;
        da.nb = nb;
        da.nv = st.nv;
        da.ds = st.ds;
        da.out_f = out_f;
        da.out_i = out_i;
        da.out_stride = out_stride;
        da.sums = sums;
        da.spread = spread;
        da.err = (int*)ctx->errflag.p;
        da.chunk_kb = ctx->tune.dedisp_kb;
        da.wait_polls = ctx->wait_polls;
        ProfScope ps(ctx, 1, s);
        PSS_CUDA(launch_dedisp(da, ctx->num_sms, s));
        return PSS_OK;
    }
    ProfScope ps(ctx, 1, s);
    DedispArgs da{};
    da.xcm = (const uint8_t*)ctx->xcm.p;
    da.pitch = pitch;
    da.ck = std::max<int32_t>(T.ckmax, 1);
    da.delays = base + T.e_off + (SB.g_lo - T.g_begin) * ck;
    da.dstride = ck;
    da.zsub = (const int2*)(base + T.z_off);
    da.nz = plan->nsub;
    da.nb = SB.ngb;
    da.nv = SB.len1;
    da.ds = 1;
    da.out_f = nullptr;
    da.out_i = (int32_t*)subu;
    da.out_stride = SB.stride1;
    da.zout = (int64_t)SB.ngb * SB.stride1;
    da.sums = nullptr;
    da.spread = SB.spread1;
    da.err = (int*)ctx->errflag.p;
    da.chunk_kb = ctx->tune.dedisp_kb;
    da.wait_polls = ctx->wait_polls;
    PSS_CUDA(launch_dedisp(da, ctx->num_sms, s));
    SubsumArgs sa{};
    sa.u = (const int32_t*)subu;
    sa.u_zstride = (int64_t)SB.ngb * SB.stride1;
    sa.u_rowstride = SB.stride1;
    sa.u_len = SB.len1;
    sa.nsub = plan->nsub;
    sa.D = base + T.d_off + (b0 - dm_begin) * plan->nsub;
    // group rows relative to the batch: (first - b0, count)
    sa.grp = (const int2*)(base + T.grp_off) + (SB.g_lo - T.g_begin);
    sa.ngrp = SB.ngb;
    sa.nb = nb;
    sa.nv = st.nv;
    sa.ds = st.ds;
    sa.wait_polls = ctx->wait_polls;
    sa.out_f = out_f;
    sa.out_i = out_i;
    sa.out_stride = out_stride;
    sa.sums = sums;
    sa.spread = SB.spread2;
    sa.b0rel = (int32_t)(b0 - dm_begin);
    sa.err = (int*)ctx->errflag.p;
    PSS_CUDA(launch_subsum(sa, s));
    return PSS_OK;
}

// Single-pulse events from raw detections: S/N = (B - w mu)/(sigma sqrt(w))
// with mu, sigma from the trial's exact moments (FP64, the order of the
// detection kernel); per trial, the detections by S/N (descending; ties:
// smaller width, then earlier) are kept when their interval [t, t + w)
// overlaps none kept before.  Output sorted by (trial, t).
void sp_prune(std::vector<SpRaw>& raw, const std::vector<unsigned long long>& mom, int64_t dm_begin, int64_t dm_end,
              const pss_plan* plan, std::vector<pss_sp_event>* out) {
    std::sort(raw.begin(), raw.end(), [](const SpRaw& a, const SpRaw& b) {
        return a.dm_idx != b.dm_idx ? a.dm_idx < b.dm_idx : (a.w != b.w ? a.w < b.w : a.t < b.t);
    });
    const int64_t nt = dm_end - dm_begin;
    std::vector<size_t> start(nt + 1, raw.size());
    for (size_t i = raw.size(); i-- > 0;) start[raw[i].dm_idx - dm_begin] = i;
    for (int64_t i = nt - 1; i >= 0; --i) start[i] = std::min(start[i], start[i + 1]);
    std::vector<std::vector<pss_sp_event>> per(nt);
    parallel_for_fn(nt, 8, [&](int64_t i) {
        const size_t a = start[i], b = start[i + 1];
        if (a == b) return;
        const double fS1 = (double)mom[2 * i], fS2 = (double)mom[2 * i + 1];
        const double fN = (double)plan->stages[plan->stage_of[dm_begin + i]].nv;
        const double mu = fS1 / fN;
        double var = (fS2 - fS1 * fS1 / fN) / fN;
        if (!(var > 0.0)) var = 0.0;
        const double sigma = sqrt(var);
        std::vector<pss_sp_event> ev;
        for (size_t k = a; k < b; ++k) {
            pss_sp_event e;
            e.dm_idx = raw[k].dm_idx;
            e.width = raw[k].w;
            e.t = raw[k].t;
            e.boxsum = raw[k].B;
            const double w = (double)raw[k].w;
            e.snr = ((double)raw[k].B - w * mu) / (sigma * sqrt(w));
            ev.push_back(e);
        }
        std::sort(ev.begin(), ev.end(), [](const pss_sp_event& x, const pss_sp_event& y) {
            if (x.snr != y.snr) return x.snr > y.snr;
            if (x.width != y.width) return x.width < y.width;
            return x.t < y.t;
        });
        std::map<int64_t, int64_t> kept;  // start -> end (exclusive), disjoint
        std::vector<pss_sp_event> keep;
        for (const auto& e : ev) {
            const int64_t s0 = e.t, s1 = e.t + e.width;
            auto it = kept.lower_bound(s0);
            if (it != kept.end() && it->first < s1) continue;
            if (it != kept.begin() && std::prev(it)->second > s0) continue;
            kept.emplace(s0, s1);
            keep.push_back(e);
        }
        std::sort(keep.begin(), keep.end(), [](const pss_sp_event& x, const pss_sp_event& y) { return x.t < y.t; });
        per[i].swap(keep);
    });
    for (auto& v : per) out->insert(out->end(), v.begin(), v.end());
}

enum Mode { MODE_SPECTRUM, MODE_PLANE, MODE_SEARCH, MODE_GAINS };

struct Outputs {
    float* spec = nullptr;   // MODE_SPECTRUM: user device buffer
    float* plane = nullptr;  // MODE_PLANE: user device buffer
    float* gains = nullptr;  // MODE_GAINS: device [trial - dm_begin][blocks]
};

pss_status check_cfg(const pss_search_cfg* cfg, const Plan& P) {
    if (!cfg) return fail(PSS_EINVAL, "null search cfg");
    if (cfg->zmax < 0) return fail(PSS_EINVAL, "zmax must be >= 0");
    if (cfg->zmax > 0) {
        if (!(cfg->dz > 0)) return fail(PSS_EINVAL, "dz must be > 0");
        const double r = cfg->zmax / cfg->dz;
        if (fabs(r - llround(r)) > 1e-9) return fail(PSS_EINVAL, "zmax must be a multiple of dz");
        if (cfg->zmax > 1200) return fail(PSS_EINVAL, "zmax above 1200 is not supported");
    }
    const int nh = cfg->numharm;
    if (nh < 1 || nh > 32 || (nh & (nh - 1))) return fail(PSS_EINVAL, "numharm must be a power of two in [1, 32]");
    const int W = cfg->whiten_block;
    if (W < 64 || W > 4096 || (W & (W - 1))) return fail(PSS_EINVAL, "whiten_block must be a power of two in [64, 4096]");
    if (cfg->halfwidth_extra < 1 || cfg->halfwidth_extra > 64)
        return fail(PSS_EINVAL, "halfwidth_extra must be in [1, 64]");
    for (const auto& st : P.stages)
        if ((st.nfft / 2) % W != 0 || st.nfft / 2 < 64)
            return fail(PSS_EINVAL, "whiten_block must divide nfft/2 (and nfft >= 128) for every stage");
    return PSS_OK;
}

int nz_of(const pss_search_cfg* cfg) { return cfg->zmax ? (int)llround(2.0 * cfg->zmax / cfg->dz) + 1 : 1; }

// Build (or reuse) the response templates of cfg in ctx->taps.
pss_status ensure_templates(pss_ctx* ctx, const pss_search_cfg* cfg, cudaStream_t s) {
    const double dz = cfg->zmax ? cfg->dz : 1.0;
    if (ctx->tap_zmax == cfg->zmax && ctx->tap_extra == cfg->halfwidth_extra && ctx->tap_dz == dz) return PSS_OK;
    const int nz = nz_of(cfg);
    std::vector<int32_t> off(2 * nz), m(nz);
    int32_t total = 0;
    for (int j = 0; j < nz; ++j) {
        const double z = cfg->zmax ? -(double)cfg->zmax + (double)j * dz : 0.0;
        m[j] = (int32_t)ceil(fabs(z) / 2.0) + cfg->halfwidth_extra;
        off[2 * j] = total;
        total += 2 * m[j];
        off[2 * j + 1] = total;
        total += 2 * m[j];
    }
    PSS_TRY(ctx->taps.ensure((size_t)total * sizeof(float2)));
    PSS_TRY(ctx->tapinfo.ensure((size_t)(2 * nz + nz + 2 * nz) * sizeof(int32_t)));
    int32_t* info = (int32_t*)ctx->tapinfo.p;
    std::vector<int32_t> hinfo(3 * nz);
    for (int i = 0; i < 2 * nz; ++i) hinfo[i] = off[i];
    for (int j = 0; j < nz; ++j) hinfo[2 * nz + j] = m[j];
    PSS_CUDA(cudaMemcpyAsync(info, hinfo.data(), hinfo.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    TemplateArgs ta;
    ta.nz = nz;
    ta.zmax = cfg->zmax;
    ta.extra = cfg->halfwidth_extra;
    ta.dz = dz;
    ta.taps = (float2*)ctx->taps.p;
    ta.tap_off = info;
    ta.tap_m = info + 2 * nz;
    ta.tap_scale = (float*)(info + 3 * nz);
    ta.total = total;
    PSS_CUDA(launch_templates(ta, s));
    // template spectra for the overlap-save plane (any spectrum of >= L bins)
    ctx->ftap_ok = false;
    if (plane_fft_usable(cfg->zmax, cfg->halfwidth_extra, PLANE_FFT_L)) {
        const int mmax = (cfg->zmax + 1) / 2 + cfg->halfwidth_extra;
        PSS_TRY(ctx->ftaps.ensure((size_t)nz * 2 * PLANE_FFT_L * sizeof(float2)));
        FftTemplateArgs fa;
        fa.nz = nz;
        fa.zmax = cfg->zmax;
        fa.extra = cfg->halfwidth_extra;
        fa.dz = dz;
        fa.tap_m = info + 2 * nz;
        fa.ftaps = (float2*)ctx->ftaps.p;
        fa.L = PLANE_FFT_L;
        fa.M0 = mmax - 1;
        PSS_CUDA(launch_fft_templates(fa, s));
        ctx->ftap_ok = true;
    }
    PSS_CUDA(cudaStreamSynchronize(s));
    ctx->tap_zmax = cfg->zmax;
    ctx->tap_extra = cfg->halfwidth_extra;
    ctx->tap_dz = dz;
    return PSS_OK;
}

// Thresholds in FP32, rounded up so that S_f >= thr_f implies S_f >= thr.
float thr_f32(int n, double sigma) {
    const double t = power_threshold(n, sigma);
    float f = (float)t;
    if ((double)f < t) f = nextafterf(f, INFINITY);
    return f;
}

// Inter-pass twiddle tables of the M-point FFT (built once per size, after
// the global twiddle table; outside any graph capture).
pss_status ensure_passtw(pss_ctx* ctx, int64_t M, int variant, cudaStream_t s) {
    for (const auto& t : ctx->passtw)
        if (t.M == M && t.variant == variant) return PSS_OK;
    int rad[4] = {0, 0, 0, 0};
    const int np = fft_pass_plan(M, variant, rad);
    if (np == 0) return fail(PSS_EINVAL, "no such FFT pass split");
    Ctx::PassTw t;
    t.M = M;
    t.variant = variant;
    t.twM = ctx->twid_n;
    int64_t total = 0, Ns = rad[0];
    for (int i = 1; i < np; ++i) {
        t.off[i] = total;
        total += (int64_t)rad[i] * Ns;
        Ns *= rad[i];
    }
    if (total > 0) {
        PSS_TRY(t.buf.ensure((size_t)total * sizeof(float2)));
        Ns = rad[0];
        for (int i = 1; i < np; ++i) {
            PSS_CUDA(launch_pass_twiddles((float2*)t.buf.p + t.off[i], (const float2*)ctx->twid.p, ctx->twid_n,
                                          rad[i], Ns, s));
            Ns *= rad[i];
        }
    }
    ctx->passtw.push_back(t);
    return PSS_OK;
}

// Point the FftArgs at the inter-pass tables of its size (ensure_passtw first).
void set_passtw(const pss_ctx* ctx, FftArgs* fa) {
    for (int i = 0; i < 4; ++i) fa->ptw[i] = nullptr;
    const int64_t M = fa->nfft / 2;
    for (const auto& t : ctx->passtw)
        if (t.M == M && t.variant == fa->fft_variant && t.buf.p)
            for (int i = 1; i < 4; ++i) fa->ptw[i] = (const float2*)t.buf.p + t.off[i];
}

// One batch of consecutive trials within a plan stage.
struct BatchDesc {
    int32_t stage;
    int64_t b0;        // first trial
    int32_t nb;        // trials
    int32_t spread;    // delay spread the dedispersion launch is sized for
    int64_t out_off;   // packed output offset (spectrum / plane modes)
    SubBatch sub;      // two-stage launch sizes
};

// Everything the kernel sequence needs, computed on the host once.
struct PathSetup {
    int32_t ck = 0;
    int64_t pitch = 0;
    SubTab sub;  // two-stage tables (sub.on false: exact dedispersion)
    int nz = 1, Z = 0, nstages = 1;
    std::vector<BatchDesc> batches;
    std::vector<HarmArgs> harm;  // per stage: thresholds and f_lo cuts
    int64_t dev_cap = 0;
};

// Trials per batch for a stage of nfft-point spectra: as many as fit in
// 6 GiB of per-trial buffers (series, three spectra, and the plane when
// searching), at most 1024 and at most the n trials there are.
// Whitening and the zmax 0 plane in one kernel (k_whiten_z0; PSS_WHITEN_Z0=0
// keeps the two kernels): zmax 0 with 2m = 32 taps, warp-pair whitening of
// 256, 512 or 1024-bin blocks.  The block scales go to the spectrum buffer,
// which the fused form does not otherwise use.
bool whiten_z0_usable(const pss_search_cfg* cfg, int whiten_form) {
    static const bool on = [] {
        const char* e = getenv("PSS_WHITEN_Z0");
        return !(e && e[0] == '0');
    }();
    const int W = cfg->whiten_block;
    return on && cfg->zmax == 0 && cfg->halfwidth_extra == 16 && whiten_form == 2 && (W == 256 || W == 512 || W == 1024);
}

int64_t batch_trials(int64_t nfft, int nz, Mode mode, int64_t n) {
    const size_t per_dm = (size_t)nfft * 4 + (size_t)(nfft / 2) * 8 * 3 +
                          ((mode == MODE_PLANE || mode == MODE_GAINS) ? 0 : (size_t)nz * nfft * 4);
    int64_t B = (int64_t)((size_t)6 << 30) / (int64_t)per_dm;
    B = std::max<int64_t>(1, std::min<int64_t>(B, 1024));
    return std::min<int64_t>(B, n);
}

// Host set-up of the path over [dm_begin, dm_end): input tables, every
// device buffer at its final size, templates and twiddles.  After this the
// kernel sequence (enqueue_path) allocates nothing and never waits on the
// host, so it can be captured into a CUDA graph.
// The last set-up of a context, reused while the request is byte-for-byte
// the same (plan, file shape and mask, search parameters, trials, mode,
// capacity, tuning) and the device tables are still the ones uploaded for it:
// the host tables, batch list and launch sizes are then not rebuilt.
struct PathCache {
    std::string key;
    uint64_t gen = 0;
    PathSetup P;
    size_t need[6] = {0, 0, 0, 0, 0, 0};
};

template <class T>
void key_put(std::string* k, const T& v) {
    k->append(reinterpret_cast<const char*>(&v), sizeof(T));
}

std::string path_key(const pss_plan* plan, const pss_fil_desc* fil, const pss_search_cfg* cfg, int64_t dm_begin,
                     int64_t dm_end, Mode mode, int64_t dev_cap, int64_t max_b, const Tune& t) {
    std::string k;
    key_put(&k, plan->id);
    key_put(&k, fil->nchan);
    key_put(&k, fil->nbits);
    key_put(&k, fil->nsamp);
    key_put(&k, fil->tsamp_s);
    key_put(&k, fil->fch0_mhz);
    key_put(&k, fil->foff_mhz);
    key_put(&k, fil->layout);
    if (fil->chan_mask) k.append(reinterpret_cast<const char*>(fil->chan_mask), (size_t)fil->nchan);
    else k.push_back('\1');
    key_put(&k, *cfg);
    key_put(&k, dm_begin);
    key_put(&k, dm_end);
    key_put(&k, (int)mode);
    key_put(&k, dev_cap);
    key_put(&k, max_b);
    k.append(reinterpret_cast<const char*>(t.fft_split), sizeof t.fft_split);
    key_put(&k, t.harm_run);
    key_put(&k, t.dedisp_kb);
    key_put(&k, t.whiten_form);
    key_put(&k, t.fused);
    key_put(&k, t.plane_form);
    return k;
}

pss_status setup_path(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const pss_search_cfg* cfg,
                      int64_t dm_begin, int64_t dm_end, Mode mode, cudaStream_t s, int64_t dev_cap, PathSetup* P,
                      int64_t max_b = 0) {
    std::string key = path_key(plan, fil, cfg, dm_begin, dm_end, mode, dev_cap, max_b, ctx->tune);
    PathCache* pc = static_cast<PathCache*>(ctx->path_cache.get());
    const bool hit = pc && pc->gen == ctx->delays_gen && pc->key == key && dm_end > dm_begin;
    if (hit) {
        *P = pc->P;
    } else {
        PSS_TRY(setup_input(ctx, plan, fil, dm_begin, dm_end, s, &P->ck, &P->pitch, &P->sub));
    }
    if (!hit) {
        P->batches.clear();
        P->harm.clear();
    }
    P->dev_cap = dev_cap;
    if (dm_end == dm_begin) return PSS_OK;
    PSS_TRY(ensure_templates(ctx, cfg, s));
    P->nz = nz_of(cfg);
    P->Z = cfg->zmax ? (int)llround(cfg->zmax / cfg->dz) : 0;
    P->nstages = (int)log2((double)cfg->numharm) + 1;
    const std::vector<int32_t> hd = (hit || P->sub.on) ? std::vector<int32_t>()
                                                       : compact_delays(plan, kept_channels(fil), dm_begin, dm_end);
    if (mode == MODE_SEARCH) {
        PSS_TRY(ctx->cands.ensure((size_t)dev_cap * sizeof(pss_raw_cand)));
        PSS_TRY(ctx->counter.ensure(sizeof(unsigned long long)));
    }
    // twiddle table covering every stage's nfft (powers of two: the largest suffices)
    int64_t nfft_max = 0;
    for (const auto& st : plan->stages) nfft_max = std::max<int64_t>(nfft_max, st.nfft);
    if (ctx->twid_n < nfft_max) {
        PSS_TRY(ctx->twid.ensure((size_t)nfft_max * sizeof(float2)));
        PSS_CUDA(launch_twiddles((float2*)ctx->twid.p, nfft_max, s));
        ctx->twid_n = nfft_max;
    }
    for (const auto& st : plan->stages)
        if (st.n_dm > 0) PSS_TRY(ensure_passtw(ctx, st.nfft / 2, ctx->tune.split_for(st.nfft / 2), s));
    size_t need_series = 0, need_fft = 0, need_sums = 0, need_plane = 0, need_subu = 0;
    int64_t out_off = 0;
    if (hit) {
        need_series = pc->need[0];
        need_fft = pc->need[1];
        need_sums = pc->need[2];
        need_plane = pc->need[3];
        need_subu = pc->need[4];
    }
    for (size_t si = 0; si < plan->stages.size() && !hit; ++si) {
        const StageInfo& st = plan->stages[si];
        const int64_t lo = std::max<int64_t>(dm_begin, st.first);
        const int64_t hi = std::min<int64_t>(dm_end, st.first + st.n_dm);
        HarmArgs ha{};
        const double T = (double)(st.nfft * (int64_t)st.ds) * plan->tsamp;
        for (int k = 0; k < P->nstages; ++k) {
            const int n = 1 << k;
            ha.thr[k] = thr_f32(n, cfg->sigma_thr);
            ha.hmin[k] = (int32_t)std::min<double>(ceil((double)(2 * n) * T * cfg->f_lo_hz), 2e9);
        }
        P->harm.push_back(ha);
        if (lo >= hi) continue;
        const int64_t nfft = st.nfft, M = nfft / 2;
        int64_t B = batch_trials(nfft, P->nz, mode, hi - lo);
        if (max_b > 0) B = std::min(B, max_b);
        // two-stage plans: whole groups per batch where possible
        if (P->sub.on && B > plan->sub_group) B = B / plan->sub_group * plan->sub_group;
        need_series = std::max(need_series, (size_t)B * nfft * 4);
        need_sums = std::max(need_sums, (size_t)B * 8);
        need_fft = std::max(need_fft, (size_t)B * M * 8);
        if (mode == MODE_SEARCH) need_plane = std::max(need_plane, (size_t)B * P->nz * nfft * 4);
        for (int64_t b0 = lo; b0 < hi; b0 += B) {
            BatchDesc d;
            d.stage = (int32_t)si;
            d.b0 = b0;
            d.nb = (int32_t)std::min<int64_t>(B, hi - b0);
            if (P->sub.on) {
                d.spread = 0;
                d.sub = sub_batch(plan, P->sub, P->ck, dm_begin, b0, d.nb, st.nv, st.ds);
                need_subu = std::max(need_subu, (size_t)plan->nsub * d.sub.ngb * d.sub.stride1 * 4 + subsum_slack_bytes(d.sub.spread2));
            } else {
                d.spread = delay_spread(hd.data() + (size_t)(b0 - dm_begin) * P->ck, d.nb, P->ck);
            }
            d.out_off = out_off;
            out_off += (mode == MODE_SPECTRUM) ? (int64_t)d.nb * M : (mode == MODE_PLANE) ? (int64_t)d.nb * P->nz * nfft : 0;
            P->batches.push_back(d);
        }
    }
    PSS_TRY(ctx->series.ensure(need_series));
    if (need_subu) PSS_TRY(ctx->subu.ensure(need_subu));
    PSS_TRY(ctx->sums.ensure(need_sums));
    PSS_TRY(ctx->fftA.ensure(need_fft));
    PSS_TRY(ctx->fftB.ensure(need_fft));
    if (mode != MODE_SPECTRUM) PSS_TRY(ctx->spec.ensure(need_fft));
    if (mode == MODE_SEARCH) PSS_TRY(ctx->plane.ensure(need_plane));
    if (!hit) {
        auto c = std::make_shared<PathCache>();
        c->key.swap(key);
        c->gen = ctx->delays_gen;
        c->P = *P;
        c->need[0] = need_series;
        c->need[1] = need_fft;
        c->need[2] = need_sums;
        c->need[3] = need_plane;
        c->need[4] = need_subu;
        ctx->path_cache = c;
    }
    return PSS_OK;
}

// The kernel sequence of the path (no allocation, no host waits): unpack,
// then per batch dedisperse, FFT + whiten, plane, harmonic sums.
pss_status enqueue_path(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const uint8_t* src,
                        const pss_search_cfg* cfg, int64_t dm_begin, const PathSetup& P, Mode mode, Outputs outs,
                        cudaStream_t s, bool snapshots = false) {
    PSS_TRY(enqueue_prep(ctx, fil, src, P.ck, P.pitch, s));
    if (P.batches.empty()) return PSS_OK;
    if (mode == MODE_SEARCH) PSS_CUDA(cudaMemsetAsync(ctx->counter.p, 0, sizeof(unsigned long long), s));
    for (const BatchDesc& d : P.batches) {
        const StageInfo& st = plan->stages[d.stage];
        const int64_t nfft = st.nfft, M = nfft / 2;
        PSS_CUDA(cudaMemsetAsync(ctx->sums.p, 0, (size_t)d.nb * 8, s));
        PSS_TRY(enqueue_dedisp(ctx, plan, P.ck, P.pitch, P.sub, st, dm_begin, d.b0, d.nb, d.spread, d.sub,
                               ctx->subu.p, (float*)ctx->series.p, nullptr, nfft,
                               (unsigned long long*)ctx->sums.p, s));
        const bool fused = (mode == MODE_SEARCH || mode == MODE_PLANE) && cfg->zmax == 0 && nfft == (int64_t(1) << 18) &&
                           cfg->whiten_block == 1024 && cfg->halfwidth_extra == 16 && ctx->tune.fused &&
                           spec_cluster_usable();
        float* plane_out = (mode == MODE_PLANE) ? outs.plane + d.out_off : (float*)ctx->plane.p;
        if (fused) {
            // FFT, whitening and the zmax 0 plane in one cluster launch (k_specfused.cu)
            SpecArgs sa;
            sa.series = (const float*)ctx->series.p;
            sa.series_stride = nfft;
            sa.sums = (const unsigned long long*)ctx->sums.p;
            sa.nv = st.nv;
            sa.nfft = nfft;
            sa.nb = d.nb;
            sa.plane = plane_out;
            sa.plane_stride = (int64_t)P.nz * nfft;
            sa.tw = (const float2*)ctx->twid.p;
            sa.twM = ctx->twid_n;
            sa.tap_scale1 = (const float*)((const int32_t*)ctx->tapinfo.p + 3 * P.nz) + 1;
            ProfScope ps(ctx, 2, s);
            PSS_CUDA(launch_spec_cluster(sa, s));
        } else {
            FftArgs fa{};
            fa.series = (const float*)ctx->series.p;
            fa.series_stride = nfft;
            fa.sums = (const unsigned long long*)ctx->sums.p;
            fa.nv = st.nv;
            fa.nfft = nfft;
            fa.nb = d.nb;
            fa.bufA = (float2*)ctx->fftA.p;
            fa.bufB = (float2*)ctx->fftB.p;
            float2* spec = (mode == MODE_SPECTRUM) ? (float2*)(outs.spec) + d.out_off : (float2*)ctx->spec.p;
            fa.spec_out = spec;
            fa.spec_stride = M;
            fa.whiten_block = cfg->whiten_block;
            fa.tw = (const float2*)ctx->twid.p;
            fa.twM = ctx->twid_n;
            fa.fft_variant = ctx->tune.split_for(M);
            fa.whiten_form = ctx->tune.whiten_form >= 0 ? ctx->tune.whiten_form : 2;
            set_passtw(ctx, &fa);
            fa.whiten = 1;
            fa.gains_out = nullptr;
            fa.gains_stride = 0;
            if (mode == MODE_GAINS) {
                fa.gains_out = outs.gains + (d.b0 - dm_begin) * (M / cfg->whiten_block);
                fa.gains_stride = M / cfg->whiten_block;
            }
            const bool z0 = (mode == MODE_SEARCH || mode == MODE_PLANE) && whiten_z0_usable(cfg, fa.whiten_form);
            if (z0) {
                fa.z0_plane = plane_out;
                fa.z0_plane_stride = (int64_t)P.nz * nfft;
                fa.z0_scale1 = (const float*)((const int32_t*)ctx->tapinfo.p + 3 * P.nz) + 1;
                fa.wscale = (float*)ctx->spec.p;
            }
            PSS_CUDA(launch_fft_whiten(fa, s, ctx));
            if (mode == MODE_SPECTRUM || mode == MODE_GAINS) continue;
            if (!z0) {
                PlaneArgs pl{};
                pl.spec = spec;
                pl.spec_stride = M;
                pl.nfft = nfft;
                pl.nb = d.nb;
                pl.plane = (mode == MODE_PLANE) ? outs.plane + d.out_off : (float*)ctx->plane.p;
                pl.plane_stride = (int64_t)P.nz * nfft;
                pl.zmax = cfg->zmax;
                pl.dz = cfg->zmax ? cfg->dz : 1.0;
                pl.extra = cfg->halfwidth_extra;
                pl.taps = (const float2*)ctx->taps.p;
                const int32_t* info = (const int32_t*)ctx->tapinfo.p;
                pl.tap_off = info;
                pl.tap_m = info + 2 * P.nz;
                pl.tap_scale = (const float*)(info + 3 * P.nz);
                pl.ftaps = nullptr;
                if (ctx->ftap_ok && plane_fft_usable(cfg->zmax, cfg->halfwidth_extra, M)) {
                    const int mmax = (cfg->zmax + 1) / 2 + cfg->halfwidth_extra;
                    pl.ftaps = (const float2*)ctx->ftaps.p;
                    pl.fL = PLANE_FFT_L;
                    pl.fM0 = mmax - 1;
                    pl.fV = PLANE_FFT_L - 2 * mmax + 1;
                    pl.tw = (const float2*)ctx->twid.p;
                    pl.twM = ctx->twid_n;
                    pl.nz = P.nz;
                    pl.form = ctx->tune.plane_form;
                    pl.zrow0 = -1;
                    for (int j = 0; j < P.nz; ++j)
                        if (-(double)cfg->zmax + (double)j * pl.dz == 0.0) pl.zrow0 = j;
                }
                {
                    ProfScope ps(ctx, 4, s);
                    PSS_CUDA(launch_plane(pl, s));
                }
            }
        }
        if (mode == MODE_PLANE) continue;
        HarmArgs ha = P.harm[d.stage];
        ha.run = ctx->tune.harm_run;
        ha.plane = plane_out;
        ha.plane_stride = (int64_t)P.nz * nfft;
        ha.nfft = nfft;
        ha.nz = P.nz;
        ha.Z = P.Z;
        ha.nb = d.nb;
        ha.dm0 = (int32_t)d.b0;
        ha.nstages = P.nstages;
        ha.out = (pss_raw_cand*)ctx->cands.p;
        ha.counter = (unsigned long long*)ctx->counter.p;
        ha.cap = P.dev_cap;
        {
            ProfScope ps(ctx, 5, s);
            PSS_CUDA(launch_harm(ha, s));
        }
        if (snapshots) {
            // detection count after this batch, then an event the host can wait on
            const size_t bi = (size_t)(&d - P.batches.data());
            PSS_CUDA(cudaMemcpyAsync(ctx->batch_cnt + bi, ctx->counter.p, sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, s));
            // under stream capture the record must be external (an event-record node the host can
            // wait on); outside capture that flag is refused
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            PSS_CUDA(cudaStreamIsCapturing(s, &cs));
            if (cs == cudaStreamCaptureStatusActive)
                PSS_CUDA(cudaEventRecordWithFlags(ctx->batch_ev[bi], s, cudaEventRecordExternal));
            else
                PSS_CUDA(cudaEventRecord(ctx->batch_ev[bi], s));
        }
    }
    return PSS_OK;
}

// Run the path over [dm_begin, dm_end) in batches within each plan stage.
pss_status run_path(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data, int on_dev,
                    const pss_search_cfg* cfg, int64_t dm_begin, int64_t dm_end, Mode mode, Outputs outs,
                    cudaStream_t s, int64_t dev_cap) {
    HostTimer tm;
    PathSetup P;
    PSS_TRY(setup_path(ctx, plan, fil, cfg, dm_begin, dm_end, mode, s, dev_cap, &P));
    const uint8_t* src = nullptr;
    PSS_TRY(upload_input(ctx, fil, data, on_dev, s, &src));
    tm.mark("setup");
    return enqueue_path(ctx, plan, fil, src, cfg, dm_begin, P, mode, outs, s);
}

}  // namespace

pss_status take_cands(const std::vector<pss_cand>& v, pss_cand* out, int64_t cap, int64_t* n_out) {
    *n_out = (int64_t)v.size();
    if ((int64_t)v.size() > cap) return fail(PSS_ECAP, "output capacity too small (count in *n_out)");
    if (!v.empty()) {
        if (!out) return fail(PSS_EINVAL, "null output buffer");
        memcpy(out, v.data(), v.size() * sizeof(pss_cand));
    }
    return PSS_OK;
}

namespace {

// A kernel's bounded wait expired since the flag was last cleared: report it
// (and clear it).
// The status a read of the error flag gives (and the flag cleared on s).
pss_status errflag_status(pss_ctx* ctx, int flag, cudaStream_t s) {
    if (flag) {
        PSS_CUDA(cudaMemsetAsync(ctx->errflag.p, 0, sizeof(int), s));
        if (flag == 1) return fail(PSS_ETIMEOUT, "a kernel's bounded wait on its staging barrier expired; results discarded");
        return fail(PSS_EINVAL, "dedispersion refused a delay spread larger than its launch was sized for; results discarded");
    }
    return PSS_OK;
}

pss_status check_errflag(pss_ctx* ctx, cudaStream_t s) {
    if (!ctx->errflag.p) return PSS_OK;
    int flag = 0;
    PSS_CUDA(cudaMemcpyAsync(&flag, ctx->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    PSS_CUDA(cudaStreamSynchronize(s));
    return errflag_status(ctx, flag, s);
}

// Trials per DM batch of a pipelined search of n trials: three batches of
// 30 % and a last one of about 10 % (at least 256 trials in all), so that
// the host sift of all but the last overlaps the device work and the sift
// left after the device finishes is short; two batches from 64 trials.  (A
// last batch of 5 % is shorter on the device than the host sift of the
// batch before it, which then ends later.)
int64_t pipeline_batch(int64_t n) { return n >= 256 ? (3 * n + 9) / 10 : (n >= 64 ? (n + 1) / 2 : 0); }

// Events and pinned count slots for n DM batches, and a stream for downloads.
pss_status ensure_snapshots(pss_ctx* ctx, int n) {
    if (!ctx->stream2) PSS_CUDA(cudaStreamCreateWithFlags(&ctx->stream2, cudaStreamNonBlocking));
    while ((int)ctx->batch_ev.size() < n) {
        cudaEvent_t e = nullptr;
        PSS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->batch_ev.push_back(e);
    }
    if (ctx->batch_cnt_n < n) {
        if (ctx->batch_cnt) cudaFreeHost(ctx->batch_cnt);
        ctx->batch_cnt = nullptr;
        ctx->batch_cnt_n = 0;
        PSS_CUDA(cudaHostAlloc((void**)&ctx->batch_cnt, (size_t)n * sizeof(unsigned long long), cudaHostAllocDefault));
        ctx->batch_cnt_n = n;
    }
    return PSS_OK;
}

pss_status ensure_raw_pinned(pss_ctx* ctx, size_t n) {
    if (ctx->raw_pinned_n >= n) return PSS_OK;
    if (ctx->raw_pinned) cudaFreeHost(ctx->raw_pinned);
    ctx->raw_pinned = nullptr;
    ctx->raw_pinned_n = 0;
    const size_t want = n + n / 4 + 4096;
    PSS_CUDA(cudaHostAlloc((void**)&ctx->raw_pinned, want * sizeof(pss_raw_cand), cudaHostAllocDefault));
    ctx->raw_pinned_n = want;
    return PSS_OK;
}

// The host side of one finished DM batch of a pipelined search: its raw
// detections sifted within their trials and the survivors added to `surv`;
// for one-row planes (zmax 0) the survivors stay ordered by r (stable merge),
// so the across-trial linkage after the last batch needs no sort; for 2-D
// planes they are linked to the earlier ones (`lk`).
pss_status absorb_batch(const pss_plan* plan, const pss_search_cfg* cfg, const pss_raw_cand* raw, int64_t n,
                        std::vector<SiftItem>* surv, SiftLinker* lk) {
    const size_t old = surv->size();
    PSS_TRY(sift_within(*plan, *cfg, raw, n, surv));
    if (cfg->zmax == 0) {
        auto by_r = [](const SiftItem& a, const SiftItem& b) { return a.kr < b.kr; };
        std::stable_sort(surv->begin() + old, surv->end(), by_r);
        std::inplace_merge(surv->begin(), surv->begin() + old, surv->end(), by_r);
    } else if (lk) {
        lk->add(*surv, old);
    }
    return PSS_OK;
}

// After the kernels of a search were enqueued with per-batch snapshots:
// wait for each DM batch in turn, download its detections on the second
// stream and run the within-trial sift on the host while the device works
// on the later batches.  *overflow: a batch's count passed `cap` (its
// detections are incomplete; the caller redoes the search larger).
pss_status drain_batches(pss_ctx* ctx, const pss_plan* plan, const pss_search_cfg* cfg, size_t nbatches,
                         int64_t cap, std::vector<SiftItem>* surv, bool* overflow, unsigned long long* total,
                         SiftLinker* lk = nullptr) {
    *overflow = false;
    unsigned long long prev = 0;
    for (size_t i = 0; i < nbatches; ++i) {
        PSS_CUDA(cudaEventSynchronize(ctx->batch_ev[i]));
        const unsigned long long cnt = ctx->batch_cnt[i];
        *total = cnt;
        if (*overflow) continue;
        if ((int64_t)cnt > cap) {
            *overflow = true;
            continue;
        }
        if (cnt > prev) {
            PSS_TRY(ensure_raw_pinned(ctx, (size_t)(cnt - prev)));
            PSS_CUDA(cudaStreamWaitEvent(ctx->stream2, ctx->batch_ev[i], 0));
            PSS_CUDA(cudaMemcpyAsync(ctx->raw_pinned, (const pss_raw_cand*)ctx->cands.p + prev,
                                     (size_t)(cnt - prev) * sizeof(pss_raw_cand), cudaMemcpyDeviceToHost,
                                     ctx->stream2));
            PSS_CUDA(cudaStreamSynchronize(ctx->stream2));
            // the batch's within-trial sift and hand-over while the device works on the later batches
            PSS_TRY(absorb_batch(plan, cfg, ctx->raw_pinned, (int64_t)(cnt - prev), surv, lk));
        }
        prev = cnt;
    }
    return PSS_OK;
}

// The whole search of [dm_begin, dm_end) with its sift.  The trials run in
// at least two DM batches so that the within-trial sift of the first ones
// overlaps the device work of the later ones.
pss_status search_pipelined(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data, int on_dev,
                            const pss_search_cfg* cfg, int64_t dm_begin, int64_t dm_end, cudaStream_t s,
                            std::vector<pss_cand>* out) {
    PSS_TRY(check_common(ctx, plan, fil, data, dm_begin, dm_end));
    PSS_TRY(check_cfg(cfg, *plan));
    out->clear();
    if (dm_end == dm_begin) return PSS_OK;
    int64_t cap = ctx->cands.bytes ? (int64_t)(ctx->cands.bytes / sizeof(pss_raw_cand)) : (int64_t)1 << 20;
    const int64_t n = dm_end - dm_begin;
    HostTimer tm;
    for (int attempt = 0; attempt < 2; ++attempt) {
        PathSetup P;
        PSS_TRY(setup_path(ctx, plan, fil, cfg, dm_begin, dm_end, MODE_SEARCH, s, cap, &P, pipeline_batch(n)));
        const uint8_t* src = nullptr;
        PSS_TRY(upload_input(ctx, fil, data, on_dev, s, &src));
        // one pinned slot per DM batch for its detection count, and one for the error flag
        const size_t nb = P.batches.size();
        PSS_TRY(ensure_snapshots(ctx, (int)nb + 1));
        PSS_TRY(enqueue_path(ctx, plan, fil, src, cfg, dm_begin, P, MODE_SEARCH, Outputs(), s, true));
        if (ctx->errflag.p)
            PSS_CUDA(cudaMemcpyAsync(ctx->batch_cnt + nb, ctx->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        tm.mark("enqueue");
        std::vector<SiftItem> surv;
        SiftLinker lk;
        bool overflow = false;
        unsigned long long total = 0;
        PSS_TRY(drain_batches(ctx, plan, cfg, nb, cap, &surv, &overflow, &total, &lk));
        PSS_CUDA(cudaStreamSynchronize(s));
        tm.mark("gpu+within");
        if (ctx->errflag.p) {
            int flag = 0;
            memcpy(&flag, ctx->batch_cnt + nb, sizeof(int));
            PSS_TRY(errflag_status(ctx, flag, s));
        }
        if (!overflow) {
            PSS_TRY(sift_across(*plan, *cfg, surv, out, cfg->zmax ? &lk : nullptr));
            tm.mark("across");
            return PSS_OK;
        }
        cap = (int64_t)total + 1024;  // overflowed the device buffer: grow and redo
    }
    return fail(PSS_ECAP, "candidate buffer overflow persisted after resizing");
}

pss_status search_raw_vec(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data, int on_dev,
                          const pss_search_cfg* cfg, int64_t dm_begin, int64_t dm_end, std::vector<pss_raw_cand>* out,
                          cudaStream_t s, bool sorted) {
    PSS_TRY(check_common(ctx, plan, fil, data, dm_begin, dm_end));
    PSS_TRY(check_cfg(cfg, *plan));
    int64_t cap = ctx->cands.bytes ? (int64_t)(ctx->cands.bytes / sizeof(pss_raw_cand)) : (int64_t)1 << 20;
    HostTimer tm;
    for (int attempt = 0; attempt < 2; ++attempt) {
        PSS_TRY(run_path(ctx, plan, fil, data, on_dev, cfg, dm_begin, dm_end, MODE_SEARCH, Outputs(), s, cap));
        tm.mark("enqueue");
        unsigned long long cnt = 0;
        if (dm_end > dm_begin)
            PSS_CUDA(cudaMemcpyAsync(&cnt, ctx->counter.p, sizeof(cnt), cudaMemcpyDeviceToHost, s));
        PSS_CUDA(cudaStreamSynchronize(s));
        tm.mark("gpu");
        PSS_TRY(check_errflag(ctx, s));
        if ((int64_t)cnt <= cap) {
            out->resize(cnt);
            if (cnt)
                PSS_CUDA(cudaMemcpyAsync(out->data(), ctx->cands.p, cnt * sizeof(pss_raw_cand),
                                         cudaMemcpyDeviceToHost, s));
            PSS_CUDA(cudaStreamSynchronize(s));
            tm.mark("download");
            if (sorted) sort_raw(out, plan->ndm());
            tm.mark("sort");
            return PSS_OK;
        }
        cap = (int64_t)cnt + 1024;  // overflowed the device buffer: grow and redo
    }
    return fail(PSS_ECAP, "candidate buffer overflow persisted after resizing");
}

// ---- multi-file search: one launch per stage over a group of files -------
//
// The files of a group may differ in channels, samples, bits, layout and DM
// plan (exact plans) and share the search parameters.  Their trials become
// rows grouped by transform length; each length class runs in batches of
// rows (batch_trials), and every batch is one launch per stage over rows of
// several files: the work-list dedispersion (items = runs of consecutive
// trials of one file and stage, one launch per kernel variant: at most 256
// kept channels or more) into float rows, the FFT passes and whitening with
// each row's own N_v, the plane, and the harmonic sums with each row's DM
// index, file index and f_lo cut.  Before the batches, one work-list launch
// unpacks every file.  The whole sequence is captured into one graph and
// launched once.  The kernels and their arithmetic are those of the
// single-file path, so every file's sorted candidate list is byte-identical
// to a search of that file alone on a context with the same launch shapes.

struct MultiRow {
    int32_t file, stage;
    int64_t trial;
};

struct MultiBatch {
    int64_t nfft;
    int32_t nrows;
    int64_t items_narrow = 0, n_narrow = 0, ctas_narrow = 0;  // byte offset in the work list, count, CTAs
    int64_t items_wide = 0, n_wide = 0, ctas_wide = 0;
    size_t shm_narrow = 0, shm_wide = 0;
    int64_t nv_rows = 0, row_dm = 0, row_file = 0, row_hmin = 0;  // byte offsets
};

struct MultiSetup {
    std::vector<int32_t> ck;
    std::vector<int64_t> pitch, fil_off, xcm_off, tab_off;  // tab_off: int32 elements into the table block
    int64_t prep_items = 0, prep_ctas = 0;                  // byte offset of the prep items, CTAs
    int64_t tab_bytes_off = 0;                              // byte offset of the table block
    std::vector<MultiBatch> batches;
    std::vector<uint8_t> work;                              // host image of ctx->mf_work
    size_t fil_bytes = 0, xcm_bytes = 0;
    size_t need_series = 0, need_sums = 0, need_fft = 0, need_plane = 0;
    int nz = 1, Z = 0, nstages = 1;
    float thr[6] = {0, 0, 0, 0, 0, 0};
};

template <class T>
int64_t work_put(std::vector<uint8_t>* w, const T* v, size_t n) {
    const int64_t off = (int64_t)((w->size() + 255) & ~size_t(255));
    w->resize((size_t)off + n * sizeof(T));
    if (n) memcpy(w->data() + off, v, n * sizeof(T));
    return off;
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Host set-up of a group: validation, layouts and the work lists (device
// pointers are formed from the buffers' addresses, which the caller has
// sized from a first, sizing-only pass: bases null).
pss_status multi_setup(const Tune& tune, int* errflag, int32_t wait_polls, const pss_search_cfg* cfg,
                       const pss_multi_file* files,
                       int32_t nfiles, const uint8_t* fil_base, const uint8_t* xcm_base, const uint8_t* work_base,
                       float* series, unsigned long long* sums, MultiSetup* M) {
    *M = MultiSetup();
    M->nz = nz_of(cfg);
    M->Z = cfg->zmax ? (int)llround(cfg->zmax / cfg->dz) : 0;
    M->nstages = 0;
    while ((1 << M->nstages) <= cfg->numharm) ++M->nstages;
    for (int k = 0; k < M->nstages; ++k) M->thr[k] = thr_f32(1 << k, cfg->sigma_thr);
    std::vector<int32_t> tab;
    std::vector<PrepItem> prep;
    for (int32_t f = 0; f < nfiles; ++f) {
        const pss_plan* plan = files[f].plan;
        const pss_fil_desc* fil = files[f].fil;
        const std::vector<int32_t> keep = kept_channels(fil);
        const int32_t ck = (int32_t)keep.size();
        const int64_t pitch = xcm_pitch(*plan, fil);
        M->ck.push_back(ck);
        M->pitch.push_back(pitch);
        M->fil_off.push_back((int64_t)M->fil_bytes);
        M->fil_bytes += align256((size_t)file_bytes(fil));
        M->xcm_off.push_back((int64_t)M->xcm_bytes);
        M->xcm_bytes += align256((size_t)ck * pitch + 64);
        M->tab_off.push_back((int64_t)tab.size());
        const std::vector<int32_t> hd = compact_delays(plan, keep, 0, plan->ndm());
        tab.insert(tab.end(), keep.begin(), keep.end());
        tab.insert(tab.end(), hd.begin(), hd.end());
        while (tab.size() % 64) tab.push_back(0);  // 256-byte steps
    }
    M->tab_bytes_off = work_put(&M->work, tab.data(), tab.size());
    const int32_t* tab_dev = work_base ? (const int32_t*)(work_base + M->tab_bytes_off) : nullptr;
    for (int32_t f = 0; f < nfiles; ++f) {
        PrepItem it{};
        it.a.src = (fil_base ? fil_base : (const uint8_t*)nullptr) + M->fil_off[f];
        it.a.nchan = files[f].fil->nchan;
        it.a.nbits = files[f].fil->nbits;
        it.a.layout = files[f].fil->layout;
        it.a.nsamp = files[f].fil->nsamp;
        it.a.keep = tab_dev ? tab_dev + M->tab_off[f] : nullptr;
        it.a.ck = M->ck[f];
        it.a.xcm = (uint8_t*)(xcm_base ? xcm_base : (const uint8_t*)nullptr) + M->xcm_off[f];
        it.a.pitch = M->pitch[f];
        it.first = M->prep_ctas;
        M->prep_ctas += prep_item_ctas(it.a, &it.gx);
        prep.push_back(it);
    }
    M->prep_items = work_put(&M->work, prep.data(), prep.size());
    // rows by transform length, longest first; within a length, file by file, trial by trial
    std::map<int64_t, std::vector<MultiRow>, std::greater<int64_t>> classes;
    for (int32_t f = 0; f < nfiles; ++f) {
        const Plan& P = *files[f].plan;
        for (size_t si = 0; si < P.stages.size(); ++si) {
            const StageInfo& st = P.stages[si];
            for (int64_t i = st.first; i < st.first + st.n_dm; ++i) classes[st.nfft].push_back({f, (int32_t)si, i});
        }
    }
    for (const auto& kv : classes) {
        const int64_t nfft = kv.first;
        const std::vector<MultiRow>& rows = kv.second;
        const int64_t B = batch_trials(nfft, M->nz, MODE_SEARCH, (int64_t)rows.size());
        M->need_series = std::max(M->need_series, (size_t)B * nfft * 4);
        M->need_sums = std::max(M->need_sums, (size_t)B * 8);
        M->need_fft = std::max(M->need_fft, (size_t)B * (nfft / 2) * 8);
        M->need_plane = std::max(M->need_plane, (size_t)B * M->nz * nfft * 4);
        for (size_t r0 = 0; r0 < rows.size(); r0 += (size_t)B) {
            const size_t r1 = std::min(rows.size(), r0 + (size_t)B);
            MultiBatch mb;
            mb.nfft = nfft;
            mb.nrows = (int32_t)(r1 - r0);
            std::vector<DedispItem> narrow, wide;
            std::vector<int64_t> nv_rows;
            std::vector<int32_t> row_dm, row_file, row_hmin;
            size_t a = r0;
            while (a < r1) {
                size_t e = a + 1;
                while (e < r1 && rows[e].file == rows[a].file && rows[e].stage == rows[a].stage &&
                       rows[e].trial == rows[e - 1].trial + 1)
                    ++e;
                const int32_t f = rows[a].file;
                const Plan& P = *files[f].plan;
                const StageInfo& st = P.stages[rows[a].stage];
                const int32_t ck = M->ck[f];
                const int32_t* hd = tab.data() + M->tab_off[f] + ck + (size_t)rows[a].trial * ck;
                DedispItem it{};
                it.a.xcm = (const uint8_t*)(xcm_base ? xcm_base : (const uint8_t*)nullptr) + M->xcm_off[f];
                it.a.pitch = M->pitch[f];
                it.a.ck = ck;
                it.a.delays = tab_dev ? tab_dev + M->tab_off[f] + ck + rows[a].trial * ck : nullptr;
                it.a.nb = (int32_t)(e - a);
                it.a.nv = st.nv;
                it.a.ds = st.ds;
                // (the sizing pass has no buffers yet: any non-null row address passes the checks)
                it.a.out_f = series ? series + (int64_t)(a - r0) * nfft : reinterpret_cast<float*>(uintptr_t(256));
                it.a.out_stride = nfft;
                it.a.sums = sums ? sums + (a - r0) : nullptr;
                it.a.spread = delay_spread(hd, (int64_t)(e - a), ck);
                it.a.err = errflag;
                it.a.chunk_kb = tune.dedisp_kb;
                it.a.wait_polls = wait_polls;
                size_t shm = 0;
                if (!dedisp_item(&it, tune.dedisp_kb, &shm))
                    return fail(PSS_EINVAL, "pss_search_multi: file " + std::to_string(f) +
                                                ": a delay spread too large for the dedispersion kernel");
                const bool w = ck > 256;
                std::vector<DedispItem>& dst = w ? wide : narrow;
                int64_t& ctas = w ? mb.ctas_wide : mb.ctas_narrow;
                size_t& mshm = w ? mb.shm_wide : mb.shm_narrow;
                it.first = ctas;
                ctas += (int64_t)it.gx * it.gy;
                mshm = std::max(mshm, shm);
                dst.push_back(it);
                const double T = (double)(st.nfft * (int64_t)st.ds) * P.tsamp;
                for (size_t r = a; r < e; ++r) {
                    nv_rows.push_back(st.nv);
                    row_dm.push_back((int32_t)rows[r].trial);
                    row_file.push_back(f);
                    for (int k = 0; k < 8; ++k)
                        row_hmin.push_back(k < M->nstages ? (int32_t)std::min<double>(
                                                                ceil((double)(2 << k) * T * cfg->f_lo_hz), 2e9)
                                                          : 0);
                }
                a = e;
            }
            mb.n_narrow = (int64_t)narrow.size();
            mb.n_wide = (int64_t)wide.size();
            mb.items_narrow = work_put(&M->work, narrow.data(), narrow.size());
            mb.items_wide = work_put(&M->work, wide.data(), wide.size());
            mb.nv_rows = work_put(&M->work, nv_rows.data(), nv_rows.size());
            mb.row_dm = work_put(&M->work, row_dm.data(), row_dm.size());
            mb.row_file = work_put(&M->work, row_file.data(), row_file.size());
            mb.row_hmin = work_put(&M->work, row_hmin.data(), row_hmin.size());
            M->batches.push_back(mb);
        }
    }
    return PSS_OK;
}

// The kernel sequence of a group (no allocation, no host waits: capturable).
pss_status multi_enqueue(pss_ctx* ctx, const pss_search_cfg* cfg, const MultiSetup& M, int64_t dev_cap,
                         cudaStream_t s) {
    const uint8_t* W = (const uint8_t*)ctx->mf_work.p;
    PSS_CUDA(cudaMemsetAsync(ctx->counter.p, 0, sizeof(unsigned long long), s));
    {
        ProfScope ps(ctx, 0, s);
        PSS_CUDA(launch_prep_multi((const PrepItem*)(W + M.prep_items), (int)M.ck.size(), M.prep_ctas, s));
    }
    for (const MultiBatch& b : M.batches) {
        const int64_t nfft = b.nfft, Mh = nfft / 2;
        PSS_CUDA(cudaMemsetAsync(ctx->sums.p, 0, (size_t)b.nrows * 8, s));
        {
            ProfScope ps(ctx, 1, s);
            PSS_CUDA(launch_dedisp_multi((const DedispItem*)(W + b.items_narrow), (int)b.n_narrow, b.ctas_narrow,
                                         b.shm_narrow, false, s));
        }
        if (b.n_wide) {
            ProfScope ps(ctx, 1, s);
            PSS_CUDA(launch_dedisp_multi((const DedispItem*)(W + b.items_wide), (int)b.n_wide, b.ctas_wide,
                                         b.shm_wide, true, s));
        }
        FftArgs fa{};
        fa.series = (const float*)ctx->series.p;
        fa.series_stride = nfft;
        fa.sums = (const unsigned long long*)ctx->sums.p;
        fa.nv = 0;
        fa.nv_rows = (const int64_t*)(W + b.nv_rows);
        fa.nfft = nfft;
        fa.nb = b.nrows;
        fa.bufA = (float2*)ctx->fftA.p;
        fa.bufB = (float2*)ctx->fftB.p;
        fa.spec_out = (float2*)ctx->spec.p;
        fa.spec_stride = Mh;
        fa.whiten_block = cfg->whiten_block;
        fa.tw = (const float2*)ctx->twid.p;
        fa.twM = ctx->twid_n;
        fa.fft_variant = ctx->tune.split_for(Mh);
        fa.whiten_form = ctx->tune.whiten_form >= 0 ? ctx->tune.whiten_form : 2;
        set_passtw(ctx, &fa);
        fa.whiten = 1;
        const bool z0 = whiten_z0_usable(cfg, fa.whiten_form);
        if (z0) {
            fa.z0_plane = (float*)ctx->plane.p;
            fa.z0_plane_stride = (int64_t)M.nz * nfft;
            fa.z0_scale1 = (const float*)((const int32_t*)ctx->tapinfo.p + 3 * M.nz) + 1;
            fa.wscale = (float*)ctx->spec.p;
        }
        PSS_CUDA(launch_fft_whiten(fa, s, ctx));
        if (!z0) {
            PlaneArgs pl{};
            pl.spec = (const float2*)ctx->spec.p;
            pl.spec_stride = Mh;
            pl.nfft = nfft;
            pl.nb = b.nrows;
            pl.plane = (float*)ctx->plane.p;
            pl.plane_stride = (int64_t)M.nz * nfft;
            pl.zmax = cfg->zmax;
            pl.dz = cfg->zmax ? cfg->dz : 1.0;
            pl.extra = cfg->halfwidth_extra;
            pl.taps = (const float2*)ctx->taps.p;
            const int32_t* info = (const int32_t*)ctx->tapinfo.p;
            pl.tap_off = info;
            pl.tap_m = info + 2 * M.nz;
            pl.tap_scale = (const float*)(info + 3 * M.nz);
            pl.ftaps = nullptr;
            if (ctx->ftap_ok && plane_fft_usable(cfg->zmax, cfg->halfwidth_extra, Mh)) {
                const int mmax = (cfg->zmax + 1) / 2 + cfg->halfwidth_extra;
                pl.ftaps = (const float2*)ctx->ftaps.p;
                pl.fL = PLANE_FFT_L;
                pl.fM0 = mmax - 1;
                pl.fV = PLANE_FFT_L - 2 * mmax + 1;
                pl.tw = (const float2*)ctx->twid.p;
                pl.twM = ctx->twid_n;
                pl.nz = M.nz;
                pl.form = ctx->tune.plane_form;
                pl.zrow0 = -1;
                for (int j = 0; j < M.nz; ++j)
                    if (-(double)cfg->zmax + (double)j * pl.dz == 0.0) pl.zrow0 = j;
            }
            {
                ProfScope ps(ctx, 4, s);
                PSS_CUDA(launch_plane(pl, s));
            }
        }
        HarmArgs ha{};
        for (int k = 0; k < 6; ++k) ha.thr[k] = M.thr[k];
        ha.run = ctx->tune.harm_run;
        ha.plane = (const float*)ctx->plane.p;
        ha.plane_stride = (int64_t)M.nz * nfft;
        ha.nfft = nfft;
        ha.nz = M.nz;
        ha.Z = M.Z;
        ha.nb = b.nrows;
        ha.dm0 = 0;
        ha.nstages = M.nstages;
        ha.out = (pss_raw_cand*)ctx->cands.p;
        ha.counter = (unsigned long long*)ctx->counter.p;
        ha.cap = dev_cap;
        ha.row_dm = (const int32_t*)(W + b.row_dm);
        ha.row_file = (const int32_t*)(W + b.row_file);
        ha.row_hmin = (const int32_t*)(W + b.row_hmin);
        {
            ProfScope ps(ctx, 5, s);
            PSS_CUDA(launch_harm(ha, s));
        }
    }
    return PSS_OK;
}

// A group's search: upload, set-up, one captured graph, sift file by file.
pss_status multi_search(pss_ctx* ctx, const pss_search_cfg* cfg, const pss_multi_file* files, int32_t nfiles,
                        int on_dev, cudaStream_t s, std::vector<pss_cand>* out, std::vector<int64_t>* counts) {
    if (nfiles < 1 || !files || !cfg) return fail(PSS_EINVAL, "pss_search_multi: no files");
    for (int32_t f = 0; f < nfiles; ++f) {
        if (!files[f].plan || !files[f].fil || !files[f].data)
            return fail(PSS_EINVAL, "pss_search_multi: null plan, descriptor or data of file " + std::to_string(f));
        if (files[f].plan->nsub > 0)
            return fail(PSS_EINVAL, "pss_search_multi: two-stage (subband) plans are not supported");
        PSS_TRY(validate_search(files[f].plan, files[f].fil, cfg));
    }
    if (!ctx->errflag.p) {
        PSS_TRY(ctx->errflag.ensure(sizeof(int)));
        PSS_CUDA(cudaMemsetAsync(ctx->errflag.p, 0, sizeof(int), s));
    }
    // sizing pass, then buffers, then the work lists with real addresses
    MultiSetup M;
    PSS_TRY(multi_setup(ctx->tune, (int*)ctx->errflag.p, ctx->wait_polls, cfg, files, nfiles, nullptr, nullptr,
                        nullptr, nullptr, nullptr, &M));
    PSS_TRY(ctx->mf_fil.ensure(M.fil_bytes));
    PSS_TRY(ctx->mf_xcm.ensure(M.xcm_bytes));
    PSS_TRY(ctx->mf_work.ensure(M.work.size() + 256));
    PSS_TRY(ctx->series.ensure(M.need_series));
    PSS_TRY(ctx->sums.ensure(M.need_sums));
    PSS_TRY(ctx->fftA.ensure(M.need_fft));
    PSS_TRY(ctx->fftB.ensure(M.need_fft));
    PSS_TRY(ctx->spec.ensure(M.need_fft));
    PSS_TRY(ctx->plane.ensure(M.need_plane));
    PSS_TRY(multi_setup(ctx->tune, (int*)ctx->errflag.p, ctx->wait_polls, cfg, files, nfiles,
                        (const uint8_t*)ctx->mf_fil.p,
                        (const uint8_t*)ctx->mf_xcm.p, (const uint8_t*)ctx->mf_work.p, (float*)ctx->series.p,
                        (unsigned long long*)ctx->sums.p, &M));
    PSS_TRY(ensure_templates(ctx, cfg, s));
    int64_t nfft_max = 0;
    for (const MultiBatch& b : M.batches) nfft_max = std::max(nfft_max, b.nfft);
    if (ctx->twid_n < nfft_max) {
        PSS_TRY(ctx->twid.ensure((size_t)nfft_max * sizeof(float2)));
        PSS_CUDA(launch_twiddles((float2*)ctx->twid.p, nfft_max, s));
        ctx->twid_n = nfft_max;
    }
    for (const MultiBatch& b : M.batches) PSS_TRY(ensure_passtw(ctx, b.nfft / 2, ctx->tune.split_for(b.nfft / 2), s));
    // inputs and work lists
    for (int32_t f = 0; f < nfiles; ++f)
        PSS_CUDA(cudaMemcpyAsync((uint8_t*)ctx->mf_fil.p + M.fil_off[f], files[f].data,
                                 (size_t)file_bytes(files[f].fil),
                                 on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    PSS_CUDA(cudaMemcpyAsync(ctx->mf_work.p, M.work.data(), M.work.size(), cudaMemcpyHostToDevice, s));
    int64_t cap = std::max<int64_t>(kBatchInitialCap, (int64_t)(ctx->cands.bytes / sizeof(pss_raw_cand)));
    std::vector<pss_raw_cand> raw;
    for (int attempt = 0; attempt < 2; ++attempt) {
        PSS_TRY(ctx->cands.ensure((size_t)cap * sizeof(pss_raw_cand)));
        PSS_TRY(ctx->counter.ensure(sizeof(unsigned long long)));
        // a group whose kernel variants this context has not run yet runs eagerly (the launchers set
        // kernel attributes and the kernels load on first use); otherwise the sequence is captured into
        // one graph and launched
        bool warm = true;
        for (const MultiBatch& b : M.batches) {
            const int64_t key = b.nfft * 4 + (b.n_wide ? 2 : 0) + (b.n_narrow ? 1 : 0);
            if (!ctx->mf_seen.count(key)) warm = false;
        }
        unsigned long long cnt = 0;
        cudaError_t e = cudaSuccess;
        if (!warm) {
            PSS_TRY(multi_enqueue(ctx, cfg, M, cap, s));
            for (const MultiBatch& b : M.batches) ctx->mf_seen.insert(b.nfft * 4 + (b.n_wide ? 2 : 0) + (b.n_narrow ? 1 : 0));
        } else {
            // captured on the context's own stream (the caller's may be the legacy default stream,
            // which cannot capture), launched on the caller's stream after its uploads
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            cudaStream_t cs = ctx->stream;
            PSS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
            pss_status st = multi_enqueue(ctx, cfg, M, cap, cs);
            e = cudaStreamEndCapture(cs, &g);
            if (st != PSS_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ge, g, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(ge, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (ge) cudaGraphExecDestroy(ge);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "pss_search_multi graph");
        }
        PSS_CUDA(cudaMemcpyAsync(&cnt, ctx->counter.p, sizeof(cnt), cudaMemcpyDeviceToHost, s));
        PSS_CUDA(cudaStreamSynchronize(s));
        ctx->mf_graphs += warm ? 1 : 0;
        PSS_TRY(check_errflag(ctx, s));
        if ((int64_t)cnt <= cap) {
            raw.resize(cnt);
            if (cnt)
                PSS_CUDA(cudaMemcpyAsync(raw.data(), ctx->cands.p, cnt * sizeof(pss_raw_cand), cudaMemcpyDeviceToHost,
                                         s));
            PSS_CUDA(cudaStreamSynchronize(s));
            break;
        }
        if (attempt == 1) return fail(PSS_ECAP, "pss_search_multi: candidate buffer overflow persisted");
        cap = (int64_t)cnt + 1024;
    }
    // file by file: sort, sift
    std::vector<std::vector<pss_raw_cand>> per(nfiles);
    for (const pss_raw_cand& c : raw) {
        if (c.reserved < 0 || c.reserved >= nfiles) return fail(PSS_EINVAL, "pss_search_multi: bad file tag");
        pss_raw_cand d = c;
        d.reserved = 0;
        per[c.reserved].push_back(d);
    }
    out->clear();
    counts->assign(nfiles, 0);
    for (int32_t f = 0; f < nfiles; ++f) {
        sort_raw(&per[f], files[f].plan->ndm());
        std::vector<pss_cand> v;
        PSS_TRY(sift(*files[f].plan, *cfg, per[f].data(), (int64_t)per[f].size(), &v));
        (*counts)[f] = (int64_t)v.size();
        out->insert(out->end(), v.begin(), v.end());
    }
    return PSS_OK;
}

}  // namespace

// Device bytes a multi-file search of these files holds (host arithmetic):
// each file's bytes, channel-major copy and delay tables, the work lists,
// and the per-row buffers of the largest batch of each transform length.
size_t multi_footprint(const std::vector<const Plan*>& plans, const std::vector<const pss_fil_desc*>& fils,
                       const pss_search_cfg* cfg) {
    const int nz = nz_of(cfg);
    size_t t = 0, work = 0, series = 0, sums = 0, fft = 0, plane = 0;
    std::map<int64_t, int64_t> rows;
    int64_t nfft_max = 0;
    for (size_t f = 0; f < plans.size(); ++f) {
        const Plan& P = *plans[f];
        int64_t ck = 0;
        for (int c = 0; c < fils[f]->nchan; ++c) ck += (!fils[f]->chan_mask || fils[f]->chan_mask[c]) ? 1 : 0;
        t += align256((size_t)file_bytes(fils[f])) + align256((size_t)ck * xcm_pitch(P, fils[f]) + 64);
        work += align256((size_t)(ck + P.ndm() * ck) * 4) + 256;
        for (const auto& st : P.stages)
            if (st.n_dm > 0) rows[st.nfft] += st.n_dm;
        // per trial at most one dedispersion item (a run of one trial) and the row arrays
        work += (size_t)P.ndm() * (sizeof(DedispItem) + 8 + 4 + 4 + 32) + 4096;
    }
    for (const auto& kv : rows) {
        const int64_t nfft = kv.first;
        const int64_t B = batch_trials(nfft, nz, MODE_SEARCH, kv.second);
        nfft_max = std::max(nfft_max, nfft);
        series = std::max(series, (size_t)B * nfft * 4);
        sums = std::max(sums, (size_t)B * 8);
        fft = std::max(fft, (size_t)B * (nfft / 2) * 8);
        plane = std::max(plane, (size_t)B * nz * nfft * 4);
        t += align256((size_t)(nfft / 2) * sizeof(float2));  // inter-pass twiddles
    }
    t += align256(work) + align256(series) + align256(sums) + 3 * align256(fft) + align256(plane) +
         align256((size_t)kBatchInitialCap * sizeof(pss_raw_cand)) + 256 + align256((size_t)nfft_max * sizeof(float2));
    const int mmax = (cfg->zmax + 1) / 2 + cfg->halfwidth_extra;
    t += align256((size_t)nz * 2 * (2 * mmax) * sizeof(float2)) + align256((size_t)5 * nz * sizeof(int32_t));
    if (cfg->zmax > 0) t += align256((size_t)nz * 2 * PLANE_FFT_L * sizeof(float2));
    return t;
}

size_t ctx_device_bytes(const pss_ctx* c);

}  // namespace pss

using namespace pss;

extern "C" {

const char* pss_version(void) { return "pss 0.1 (sm_103a)"; }

pss_status pss_ctx_create(int device, pss_ctx** out) {
    if (!out) return fail(PSS_EINVAL, "pss_ctx_create: null out");
    *out = nullptr;
    int n = 0;
    PSS_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(PSS_EINVAL, "pss_ctx_create: no such device");
    PSS_CUDA(cudaSetDevice(device));
    pss_ctx* c = new pss_ctx();
    c->device = device;
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaStreamCreate");
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    // PSS_FUSED=1: the cluster-fused FFT / whitening / plane kernel where it applies
    if (const char* f = getenv("PSS_FUSED")) c->tune.fused = f[0] == '1';
    // PSS_PLANE_FORM=0 / 1: the radix 8-8-8-4 / 16-16-8 overlap-save plane kernel
    if (const char* f = getenv("PSS_PLANE_FORM")) c->tune.plane_form = f[0] == '1';
    // PSS_DEDISP_BX_MIN=k: rows with ds >= k use the boxcar-table dedispersion (0: never)
    if (const char* f = getenv("PSS_DEDISP_BX_MIN")) c->tune.bx_min = std::max(0, atoi(f));
    // PSS_DEDISP_KB=k: shared memory (KiB) for the dedispersion kernel's staged channel chunks
    if (const char* f = getenv("PSS_DEDISP_KB")) c->tune.dedisp_kb = std::min(200, std::max(16, atoi(f)));
    // PSS_WHITEN_FORM=0 / 1 / 2: block per CTA / warp per block / warp pair per block
    if (const char* f = getenv("PSS_WHITEN_FORM")) c->tune.whiten_form = (f[0] >= '0' && f[0] <= '2') ? f[0] - '0' : -1;
    *out = c;
    return PSS_OK;
}

void pss_ctx_destroy(pss_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    DevBuf* bufs[] = {&c->fil_dev, &c->xcm, &c->delays_dev, &c->subu, &c->sp_series, &c->sp_mom, &c->sp_ev,
                      &c->fold_buf, &c->bx, &c->mf_fil, &c->mf_xcm, &c->mf_work, &c->series, &c->sums, &c->fftA, &c->fftB,
                      &c->spec, &c->plane, &c->cands, &c->counter, &c->taps, &c->ftaps, &c->tapinfo, &c->errflag,
                      &c->twid, &c->chan_spec, &c->refine_gains, &c->refine_dtau, &c->refine_pts, &c->refine_out};
    for (DevBuf* b : bufs) b->release();
    for (auto& t : c->passtw) t.buf.release();
    for (cudaEvent_t e : c->batch_ev) cudaEventDestroy(e);
    if (c->batch_cnt) cudaFreeHost(c->batch_cnt);
    if (c->raw_pinned) cudaFreeHost(c->raw_pinned);
    if (c->stream2) cudaStreamDestroy(c->stream2);
    for (auto& r : c->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->prof_pool) cudaEventDestroy(e);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

pss_status pss_ctx_set_wait_limit(pss_ctx* ctx, int32_t polls) {
    if (!ctx || polls < 0) return fail(PSS_EINVAL, "pss_ctx_set_wait_limit: null ctx or negative polls");
    ctx->wait_polls = polls;
    return PSS_OK;
}

void pss_debug_fail_alloc(int64_t n) { g_alloc_countdown.store(n > 0 ? n : 0); }

pss_status pss_ctx_check(pss_ctx* ctx, void* stream) {
    if (!ctx) return fail(PSS_EINVAL, "pss_ctx_check: null ctx");
    PSS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = pick_stream(ctx, stream);
    PSS_CUDA(cudaStreamSynchronize(s));
    return check_errflag(ctx, s);
}

pss_status pss_ctx_profile(pss_ctx* ctx, int enable) {
    if (!ctx) return fail(PSS_EINVAL, "pss_ctx_profile: null ctx");
    PSS_CUDA(cudaSetDevice(ctx->device));
    for (auto& r : ctx->prof_recs) {
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_recs.clear();
    ctx->prof_on = enable != 0;
    return PSS_OK;
}

pss_status pss_ctx_profile_read(pss_ctx* ctx, double* ms, int64_t* launches) {
    if (!ctx || !ms || !launches) return fail(PSS_EINVAL, "pss_ctx_profile_read: null argument");
    PSS_CUDA(cudaSetDevice(ctx->device));
    for (int i = 0; i < PSS_NPROF_STAGES; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    for (auto& r : ctx->prof_recs) {
        PSS_CUDA(cudaEventSynchronize(r.b));
        float t = 0.f;
        PSS_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
        ms[r.stage] += t;
        launches[r.stage] += 1;
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_recs.clear();
    return PSS_OK;
}

pss_status pss_dd_plan(const pss_fil_desc* fil, const pss_dd_stage* stages, int nstages, pss_plan** out) {
    if (!out) return fail(PSS_EINVAL, "pss_dd_plan: null out");
    *out = nullptr;
    pss_plan* p = new pss_plan();
    pss_status st = build_plan(fil, stages, nstages, p);
    if (st != PSS_OK) {
        delete p;
        return st;
    }
    *out = p;
    return PSS_OK;
}

pss_status pss_dd_plan_subband(const pss_fil_desc* fil, const pss_dd_stage* stages, int nstages, int32_t nsub,
                               int32_t group, pss_plan** out) {
    if (!out) return fail(PSS_EINVAL, "pss_dd_plan_subband: null out");
    *out = nullptr;
    pss_plan* p = new pss_plan();
    pss_status st = build_plan(fil, stages, nstages, p);
    if (st == PSS_OK) st = build_subband(p, nsub, group);
    if (st != PSS_OK) {
        delete p;
        return st;
    }
    *out = p;
    return PSS_OK;
}

pss_status pss_plan_subband_info(const pss_plan* plan, int32_t* nsub, int32_t* group, int64_t* ngroups,
                                 double* group_dm, int32_t* chan_delays, int32_t* sub_delays) {
    if (!plan) return fail(PSS_EINVAL, "pss_plan_subband_info: null plan");
    if (nsub) *nsub = plan->nsub;
    if (group) *group = plan->sub_group;
    if (ngroups) *ngroups = (int64_t)plan->grp_first.size();
    if (group_dm) memcpy(group_dm, plan->grp_dm.data(), sizeof(double) * plan->grp_dm.size());
    if (chan_delays) memcpy(chan_delays, plan->sub_e.data(), sizeof(int32_t) * plan->sub_e.size());
    if (sub_delays) memcpy(sub_delays, plan->sub_D.data(), sizeof(int32_t) * plan->sub_D.size());
    return PSS_OK;
}

pss_status pss_plan_info(const pss_plan* plan, int64_t* ndm, int64_t* max_delay, double* dms, int32_t* delays) {
    if (!plan) return fail(PSS_EINVAL, "pss_plan_info: null plan");
    if (ndm) *ndm = plan->ndm();
    if (max_delay) *max_delay = plan->max_delay;
    if (dms) memcpy(dms, plan->dms.data(), sizeof(double) * plan->dms.size());
    if (delays) memcpy(delays, plan->delays.data(), sizeof(int32_t) * plan->delays.size());
    return PSS_OK;
}

pss_status pss_plan_trial_info(const pss_plan* plan, int64_t dm_idx, int32_t* stage, int64_t* nv, int64_t* nfft,
                               int32_t* ds) {
    if (!plan) return fail(PSS_EINVAL, "pss_plan_trial_info: null plan");
    if (dm_idx < 0 || dm_idx >= plan->ndm()) return fail(PSS_EINVAL, "pss_plan_trial_info: dm_idx out of range");
    const int s = plan->stage_of[dm_idx];
    const StageInfo& si = plan->stages[s];
    if (stage) *stage = s;
    if (nv) *nv = si.nv;
    if (nfft) *nfft = si.nfft;
    if (ds) *ds = si.ds;
    return PSS_OK;
}

void pss_plan_free(pss_plan* plan) { delete plan; }

pss_status pss_dedisperse(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data,
                          int data_on_device, int64_t dm_begin, int64_t dm_end, int32_t* out, void* stream) {
    PSS_TRY(check_common(ctx, plan, fil, data, dm_begin, dm_end));
    if (!out && dm_end > dm_begin) return fail(PSS_EINVAL, "pss_dedisperse: null out");
    PSS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = pick_stream(ctx, stream);
    int32_t ck = 0;
    int64_t pitch = 0;
    SubTab T;
    PSS_TRY(stage_input(ctx, plan, fil, data, data_on_device, dm_begin, dm_end, s, &ck, &pitch, &T));
    const std::vector<int32_t> hd = T.on ? std::vector<int32_t>() : compact_delays(plan, kept_channels(fil), dm_begin, dm_end);
    int64_t off = 0;
    for (size_t si = 0; si < plan->stages.size(); ++si) {
        const StageInfo& st = plan->stages[si];
        const int64_t lo = std::max<int64_t>(dm_begin, st.first);
        const int64_t hi = std::min<int64_t>(dm_end, st.first + st.n_dm);
        if (lo >= hi) continue;
        int64_t B = 1024;
        if (T.on) B = std::max<int64_t>(1, std::min<int64_t>(B, 256 / plan->sub_group) * plan->sub_group);
        for (int64_t b0 = lo; b0 < hi; b0 += B) {
            const int32_t nb = (int32_t)std::min<int64_t>(B, hi - b0);
            int32_t spread = 0;
            SubBatch SB;
            if (T.on) {
                SB = sub_batch(plan, T, ck, dm_begin, b0, nb, st.nv, st.ds);
                PSS_TRY(ctx->subu.ensure((size_t)plan->nsub * SB.ngb * SB.stride1 * 4 + subsum_slack_bytes(SB.spread2)));
            } else {
                spread = delay_spread(hd.data() + (size_t)(b0 - dm_begin) * ck, nb, ck);
            }
            PSS_TRY(enqueue_dedisp(ctx, plan, ck, pitch, T, st, dm_begin, b0, nb, spread, SB, ctx->subu.p, nullptr,
                                   out + off, st.nv, nullptr, s));
            off += (int64_t)nb * st.nv;
        }
    }
    return PSS_OK;
}

pss_status pss_single_pulse(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data,
                            int data_on_device, int64_t dm_begin, int64_t dm_end, const int32_t* widths,
                            int32_t nwidths, double sigma_thr, pss_sp_event* out, int64_t cap, int64_t* n_out,
                            void* stream) {
    if (!n_out) return fail(PSS_EINVAL, "pss_single_pulse: null n_out");
    *n_out = 0;
    PSS_TRY(check_common(ctx, plan, fil, data, dm_begin, dm_end));
    if (!widths || nwidths < 1 || nwidths > SP_MAXW)
        return fail(PSS_EINVAL, "pss_single_pulse: 1 to 32 widths are required");
    int32_t wmax = 0;
    for (int i = 0; i < nwidths; ++i) {
        if (widths[i] < 1 || widths[i] > SP_MAXWIDTH) return fail(PSS_EINVAL, "pss_single_pulse: widths must be in [1, 1024]");
        wmax = std::max(wmax, widths[i]);
    }
    if (!std::isfinite(sigma_thr)) return fail(PSS_EINVAL, "pss_single_pulse: sigma_thr must be finite");
    if (!out && cap > 0) return fail(PSS_EINVAL, "pss_single_pulse: null out");
    PSS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = pick_stream(ctx, stream);
    int32_t ck = 0;
    int64_t pitch = 0;
    SubTab T;
    PSS_TRY(stage_input(ctx, plan, fil, data, data_on_device, dm_begin, dm_end, s, &ck, &pitch, &T));
    const std::vector<int32_t> hd = T.on ? std::vector<int32_t>() : compact_delays(plan, kept_channels(fil), dm_begin, dm_end);
    PSS_TRY(ctx->counter.ensure(sizeof(unsigned long long)));
    int64_t devcap = std::max<int64_t>((int64_t)ctx->sp_ev.bytes / (int64_t)sizeof(SpRaw), 1 << 16);
    PSS_TRY(ctx->sp_ev.ensure((size_t)devcap * sizeof(SpRaw)));
    std::vector<SpRaw> raw;
    std::vector<unsigned long long> mom_all((size_t)2 * (dm_end - dm_begin));
    for (size_t si = 0; si < plan->stages.size(); ++si) {
        const StageInfo& st = plan->stages[si];
        const int64_t lo = std::max<int64_t>(dm_begin, st.first);
        const int64_t hi = std::min<int64_t>(dm_end, st.first + st.n_dm);
        if (lo >= hi) continue;
        // trials per batch: up to 1 GiB of int32 series, whole groups for two-stage plans
        int64_t B = std::max<int64_t>(1, std::min<int64_t>(1024, ((int64_t)1 << 28) / st.nv));
        if (T.on && B > plan->sub_group) B = B / plan->sub_group * plan->sub_group;
        PSS_TRY(ctx->sp_series.ensure((size_t)std::min<int64_t>(B, hi - lo) * st.nv * sizeof(int32_t)));
        PSS_TRY(ctx->sp_mom.ensure((size_t)(2 + SP_MAXW) * std::min<int64_t>(B, hi - lo) * sizeof(unsigned long long)));
        for (int64_t b0 = lo; b0 < hi; b0 += B) {
            const int32_t nb = (int32_t)std::min<int64_t>(B, hi - b0);
            int32_t spread = 0;
            SubBatch SB;
            if (T.on) {
                SB = sub_batch(plan, T, ck, dm_begin, b0, nb, st.nv, st.ds);
                PSS_TRY(ctx->subu.ensure((size_t)plan->nsub * SB.ngb * SB.stride1 * 4 + subsum_slack_bytes(SB.spread2)));
            } else {
                spread = delay_spread(hd.data() + (size_t)(b0 - dm_begin) * ck, nb, ck);
            }
            int32_t* ser = (int32_t*)ctx->sp_series.p;
            PSS_TRY(enqueue_dedisp(ctx, plan, ck, pitch, T, st, dm_begin, b0, nb, spread, SB, ctx->subu.p, nullptr,
                                   ser, st.nv, nullptr, s));
            unsigned long long* m1 = (unsigned long long*)ctx->sp_mom.p;
            unsigned long long* m2 = m1 + nb;
            PSS_CUDA(cudaMemsetAsync(m1, 0, (size_t)2 * nb * sizeof(unsigned long long), s));
            PSS_CUDA(cudaMemsetAsync(ctx->counter.p, 0, sizeof(unsigned long long), s));
            SpArgs sa{};
            sa.series = ser;
            sa.stride = st.nv;
            sa.n = st.nv;
            sa.nb = nb;
            sa.dm0 = (int32_t)b0;
            for (int i = 0; i < nwidths; ++i) sa.w[i] = widths[i];
            sa.nw = nwidths;
            sa.wmax = wmax;
            sa.thr = sigma_thr;
            sa.s1 = m1;
            sa.s2 = m2;
            sa.thr_tab = (long long*)(m2 + nb);
            // a sample sums at most 255 (8-bit) or 1 (1-bit) per kept channel and native sample
            sa.max_value = (long long)ck * (fil->nbits == 8 ? 255 : 1) * st.ds;
            sa.out = (SpRaw*)ctx->sp_ev.p;
            sa.count = (unsigned long long*)ctx->counter.p;
            sa.cap = devcap;
            PSS_CUDA(launch_single_pulse(sa, m1, m2, s));
            unsigned long long cnt = 0;
            PSS_CUDA(cudaMemcpyAsync(&cnt, ctx->counter.p, sizeof(cnt), cudaMemcpyDeviceToHost, s));
            PSS_CUDA(cudaStreamSynchronize(s));
            PSS_TRY(check_errflag(ctx, s));
            if ((int64_t)cnt > devcap) {
                // grow and detect again (the series and moments are still on the device)
                devcap = (int64_t)cnt + cnt / 4;
                PSS_TRY(ctx->sp_ev.ensure((size_t)devcap * sizeof(SpRaw)));
                sa.out = (SpRaw*)ctx->sp_ev.p;
                sa.cap = devcap;
                PSS_CUDA(cudaMemsetAsync(ctx->counter.p, 0, sizeof(unsigned long long), s));
                PSS_CUDA(launch_sp_detect_only(sa, s));
                PSS_CUDA(cudaMemcpyAsync(&cnt, ctx->counter.p, sizeof(cnt), cudaMemcpyDeviceToHost, s));
                PSS_CUDA(cudaStreamSynchronize(s));
            }
            const size_t r0 = raw.size();
            raw.resize(r0 + (size_t)cnt);
            if (cnt)
                PSS_CUDA(cudaMemcpyAsync(raw.data() + r0, ctx->sp_ev.p, (size_t)cnt * sizeof(SpRaw),
                                         cudaMemcpyDeviceToHost, s));
            PSS_CUDA(cudaMemcpyAsync(mom_all.data() + 2 * (b0 - dm_begin), m1, (size_t)nb * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, s));
            PSS_CUDA(cudaMemcpyAsync(mom_all.data() + 2 * (b0 - dm_begin) + nb, m2, (size_t)nb * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, s));
            PSS_CUDA(cudaStreamSynchronize(s));
            // moments were stored as [S1 of the batch][S2 of the batch]; reorder to per-trial pairs below
            std::vector<unsigned long long> tmp(mom_all.begin() + 2 * (b0 - dm_begin),
                                                mom_all.begin() + 2 * (b0 - dm_begin) + 2 * nb);
            for (int32_t i = 0; i < nb; ++i) {
                mom_all[2 * (b0 - dm_begin + i)] = tmp[i];
                mom_all[2 * (b0 - dm_begin + i) + 1] = tmp[nb + i];
            }
        }
    }
    // host: S/N in FP64 and greedy pruning per trial, in the oracle's order
    std::vector<pss_sp_event> events;
    sp_prune(raw, mom_all, dm_begin, dm_end, plan, &events);
    *n_out = (int64_t)events.size();
    if ((int64_t)events.size() > cap) return fail(PSS_ECAP, "pss_single_pulse: more events than cap (n_out holds the count)");
    if (!events.empty()) memcpy(out, events.data(), events.size() * sizeof(pss_sp_event));
    return PSS_OK;
}

pss_status pss_fold(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data, int data_on_device,
                    const pss_fold_req* reqs, int64_t n, int32_t nbin, int32_t nfreq, double step_bins,
                    int64_t* profiles, int64_t* counts, pss_fold_result* results, void* stream) {
    if (n < 0 || (n > 0 && (!reqs || !profiles || !counts || !results)))
        return fail(PSS_EINVAL, "pss_fold: null argument");
    if (nbin < 2 || nbin > 1024) return fail(PSS_EINVAL, "pss_fold: nbin must be in [2, 1024]");
    if (nfreq < 1 || nfreq > 64) return fail(PSS_EINVAL, "pss_fold: nfreq must be in [1, 64]");
    if (!std::isfinite(step_bins)) return fail(PSS_EINVAL, "pss_fold: step_bins must be finite");
    if (n == 0) return PSS_OK;
    int64_t lo_dm = INT64_MAX, hi_dm = -1;
    for (int64_t i = 0; i < n; ++i) {
        if (!std::isfinite(reqs[i].f_hz) || !std::isfinite(reqs[i].fdot_hz_s))
            return fail(PSS_EINVAL, "pss_fold: non-finite frequency");
        lo_dm = std::min<int64_t>(lo_dm, reqs[i].dm_idx);
        hi_dm = std::max<int64_t>(hi_dm, reqs[i].dm_idx);
    }
    PSS_TRY(check_common(ctx, plan, fil, data, lo_dm, hi_dm + 1));
    PSS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = pick_stream(ctx, stream);
    int32_t ck = 0;
    int64_t pitch = 0;
    SubTab T;
    PSS_TRY(stage_input(ctx, plan, fil, data, data_on_device, lo_dm, hi_dm + 1, s, &ck, &pitch, &T));
    const std::vector<int32_t> hd = T.on ? std::vector<int32_t>() : compact_delays(plan, kept_channels(fil), lo_dm, hi_dm + 1);
    // requests by trial; chunks of at most 256 series rows
    std::vector<int64_t> order(n);
    for (int64_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return reqs[a].dm_idx < reqs[b].dm_idx; });
    int64_t nv_max = 0;
    for (const auto& st : plan->stages) nv_max = std::max<int64_t>(nv_max, st.nv);
    constexpr int64_t MAXROWS = 256;
    PSS_TRY(ctx->sp_series.ensure((size_t)MAXROWS * nv_max * sizeof(int32_t)));
    PSS_TRY(ctx->sp_mom.ensure((size_t)2 * MAXROWS * sizeof(unsigned long long)));
    size_t q0 = 0;
    while (q0 < order.size()) {
        // runs of trials (same stage, gaps of at most 15 trials dedispersed as well) up to MAXROWS rows
        struct Run { int64_t a, b; int32_t row0; };
        std::vector<Run> runs;
        int32_t rows = 0;
        size_t q = q0;
        while (q < order.size()) {
            const int64_t d = reqs[order[q]].dm_idx;
            if (!runs.empty() && d < runs.back().b) { ++q; continue; }
            if (!runs.empty() && plan->stage_of[d] == plan->stage_of[runs.back().a] && d - runs.back().b <= 15 &&
                rows + (d + 1 - runs.back().b) <= MAXROWS) {
                rows += (int32_t)(d + 1 - runs.back().b);
                runs.back().b = d + 1;
            } else if (rows + 1 <= MAXROWS) {
                runs.push_back({d, d + 1, rows});
                rows += 1;
            } else {
                break;
            }
            ++q;
        }
        int32_t* ser = (int32_t*)ctx->sp_series.p;
        unsigned long long* m1 = (unsigned long long*)ctx->sp_mom.p;
        unsigned long long* m2 = m1 + MAXROWS;
        PSS_CUDA(cudaMemsetAsync(m1, 0, (size_t)2 * MAXROWS * sizeof(unsigned long long), s));
        for (const Run& r : runs) {
            const StageInfo& st = plan->stages[plan->stage_of[r.a]];
            const int32_t nb = (int32_t)(r.b - r.a);
            int32_t spread = 0;
            SubBatch SB;
            if (T.on) {
                SB = sub_batch(plan, T, ck, lo_dm, r.a, nb, st.nv, st.ds);
                PSS_TRY(ctx->subu.ensure((size_t)plan->nsub * SB.ngb * SB.stride1 * 4 + subsum_slack_bytes(SB.spread2)));
            } else {
                spread = delay_spread(hd.data() + (size_t)(r.a - lo_dm) * ck, nb, ck);
            }
            int32_t* out = ser + (int64_t)r.row0 * nv_max;
            PSS_TRY(enqueue_dedisp(ctx, plan, ck, pitch, T, st, lo_dm, r.a, nb, spread, SB, ctx->subu.p, nullptr, out,
                                   nv_max, nullptr, s));
            PSS_CUDA(launch_sp_moments(out, nv_max, st.nv, nb, m1 + r.row0, m2 + r.row0, s));
        }
        std::vector<unsigned long long> mom((size_t)2 * MAXROWS);
        PSS_CUDA(cudaMemcpyAsync(mom.data(), m1, mom.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        PSS_CUDA(cudaStreamSynchronize(s));
        PSS_TRY(check_errflag(ctx, s));
        // items of this chunk's requests
        std::vector<FoldItem> items;
        std::vector<int64_t> which;
        for (size_t k = q0; k < q; ++k) {
            const pss_fold_req& rq = reqs[order[k]];
            int32_t row = -1;
            for (const Run& r : runs)
                if (rq.dm_idx >= r.a && rq.dm_idx < r.b) row = r.row0 + (int32_t)(rq.dm_idx - r.a);
            const StageInfo& st = plan->stages[plan->stage_of[rq.dm_idx]];
            FoldItem it{};
            it.row = row;
            it.n = st.nv;
            it.dt = (double)st.ds * plan->tsamp;
            it.T = plan->t_span(rq.dm_idx);
            it.f = rq.f_hz;
            it.fdot = rq.fdot_hz_s;
            it.s1 = mom[row];
            it.s2 = mom[MAXROWS + row];
            items.push_back(it);
            which.push_back(order[k]);
        }
        const int64_t ni = (int64_t)items.size();
        const size_t o_items = 0, o_prof = (ni * sizeof(FoldItem) + 255) / 256 * 256;
        const size_t o_cnt = o_prof + (size_t)ni * nfreq * nbin * 8, o_chi = o_cnt + (size_t)ni * nfreq * nbin * 8;
        const size_t o_frq = o_chi + (size_t)ni * nfreq * 8, total = o_frq + (size_t)ni * nfreq * 8;
        PSS_TRY(ctx->fold_buf.ensure(total));
        char* fb = (char*)ctx->fold_buf.p;
        PSS_CUDA(cudaMemcpyAsync(fb + o_items, items.data(), ni * sizeof(FoldItem), cudaMemcpyHostToDevice, s));
        FoldArgs fa{};
        fa.series = ser;
        fa.stride = nv_max;
        fa.items = (const FoldItem*)(fb + o_items);
        fa.nbin = nbin;
        fa.nfreq = nfreq;
        fa.step_bins = step_bins;
        fa.prof = (long long*)(fb + o_prof);
        fa.counts = (long long*)(fb + o_cnt);
        fa.chi2 = (double*)(fb + o_chi);
        fa.freq = (double*)(fb + o_frq);
        PSS_CUDA(launch_fold(fa, ni, s));
        std::vector<char> host(total - o_prof);
        PSS_CUDA(cudaMemcpyAsync(host.data(), fb + o_prof, host.size(), cudaMemcpyDeviceToHost, s));
        PSS_CUDA(cudaStreamSynchronize(s));
        const long long* hp = (const long long*)host.data();
        const long long* hc = (const long long*)(host.data() + (o_cnt - o_prof));
        const double* hchi = (const double*)(host.data() + (o_chi - o_prof));
        const double* hfrq = (const double*)(host.data() + (o_frq - o_prof));
        for (int64_t i = 0; i < ni; ++i) {
            int best = 0;
            for (int k = 1; k < nfreq; ++k)
                if (hchi[i * nfreq + k] > hchi[i * nfreq + best]) best = k;
            const int64_t w = which[i];
            results[w].f_hz = hfrq[i * nfreq + best];
            results[w].chi2_red = hchi[i * nfreq + best];
            results[w].best = best;
            results[w].reserved = 0;
            memcpy(profiles + w * nbin, hp + (i * nfreq + best) * nbin, (size_t)nbin * 8);
            memcpy(counts + w * nbin, hc + (i * nfreq + best) * nbin, (size_t)nbin * 8);
        }
        q0 = q;
    }
    return PSS_OK;
}

pss_status pss_spectrum(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data,
                        int data_on_device, const pss_search_cfg* cfg, int64_t dm_begin, int64_t dm_end, float* out,
                        void* stream) {
    PSS_TRY(check_common(ctx, plan, fil, data, dm_begin, dm_end));
    PSS_TRY(check_cfg(cfg, *plan));
    if (!out && dm_end > dm_begin) return fail(PSS_EINVAL, "pss_spectrum: null out");
    PSS_CUDA(cudaSetDevice(ctx->device));
    Outputs o;
    o.spec = out;
    return run_path(ctx, plan, fil, data, data_on_device, cfg, dm_begin, dm_end, MODE_SPECTRUM, o,
                    pick_stream(ctx, stream), 0);
}

pss_status pss_power_plane(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data,
                           int data_on_device, const pss_search_cfg* cfg, int64_t dm_begin, int64_t dm_end,
                           float* out, void* stream) {
    PSS_TRY(check_common(ctx, plan, fil, data, dm_begin, dm_end));
    PSS_TRY(check_cfg(cfg, *plan));
    if (!out && dm_end > dm_begin) return fail(PSS_EINVAL, "pss_power_plane: null out");
    PSS_CUDA(cudaSetDevice(ctx->device));
    Outputs o;
    o.plane = out;
    return run_path(ctx, plan, fil, data, data_on_device, cfg, dm_begin, dm_end, MODE_PLANE, o,
                    pick_stream(ctx, stream), 0);
}

pss_status pss_search_raw(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data,
                          int data_on_device, const pss_search_cfg* cfg, int64_t dm_begin, int64_t dm_end,
                          pss_raw_cand* out, int64_t cap, int64_t* n_out, void* stream) {
    if (!n_out) return fail(PSS_EINVAL, "pss_search_raw: null n_out");
    *n_out = 0;
    if (ctx) PSS_CUDA(cudaSetDevice(ctx->device));
    std::vector<pss_raw_cand> v;
    PSS_TRY(search_raw_vec(ctx, plan, fil, data, data_on_device, cfg, dm_begin, dm_end, &v,
                           ctx ? pick_stream(ctx, stream) : nullptr, true));
    *n_out = (int64_t)v.size();
    if ((int64_t)v.size() > cap) return fail(PSS_ECAP, "pss_search_raw: output capacity too small");
    if (!v.empty()) {
        if (!out) return fail(PSS_EINVAL, "pss_search_raw: null out");
        memcpy(out, v.data(), v.size() * sizeof(pss_raw_cand));
    }
    return PSS_OK;
}

pss_status pss_sift(const pss_plan* plan, const pss_search_cfg* cfg, const pss_raw_cand* raw, int64_t n_raw,
                    pss_cand* out, int64_t cap, int64_t* n_out) {
    if (!plan || !cfg || !n_out || (n_raw > 0 && !raw)) return fail(PSS_EINVAL, "pss_sift: null argument");
    *n_out = 0;
    if (cfg->zmax > 0 && !(cfg->dz > 0)) return fail(PSS_EINVAL, "pss_sift: dz must be > 0");
    std::vector<pss_cand> v;
    PSS_TRY(sift(*plan, *cfg, raw, n_raw, &v));
    *n_out = (int64_t)v.size();
    if ((int64_t)v.size() > cap) return fail(PSS_ECAP, "pss_sift: output capacity too small");
    if (!v.empty()) {
        if (!out) return fail(PSS_EINVAL, "pss_sift: null out");
        memcpy(out, v.data(), v.size() * sizeof(pss_cand));
    }
    return PSS_OK;
}

pss_status pss_sift_in_batches(const pss_plan* plan, const pss_search_cfg* cfg, const pss_raw_cand* raw,
                               int64_t n_raw, const int64_t* dm_bounds, int32_t nbatches, pss_cand* out, int64_t cap,
                               int64_t* n_out) {
    if (!plan || !cfg || !n_out || (n_raw > 0 && !raw) || nbatches < 1 || !dm_bounds)
        return fail(PSS_EINVAL, "pss_sift_in_batches: null argument or no batch");
    *n_out = 0;
    if (cfg->zmax > 0 && !(cfg->dz > 0)) return fail(PSS_EINVAL, "pss_sift_in_batches: dz must be > 0");
    for (int32_t b = 0; b < nbatches; ++b)
        if (dm_bounds[b] > dm_bounds[b + 1]) return fail(PSS_EINVAL, "pss_sift_in_batches: DM bounds must not decrease");
    std::vector<SiftItem> surv;
    SiftLinker lk;
    std::vector<pss_raw_cand> part;
    for (int32_t b = 0; b < nbatches; ++b) {
        part.clear();
        for (int64_t i = 0; i < n_raw; ++i)
            if (raw[i].dm_idx >= dm_bounds[b] && raw[i].dm_idx < dm_bounds[b + 1]) part.push_back(raw[i]);
        PSS_TRY(absorb_batch(plan, cfg, part.data(), (int64_t)part.size(), &surv, &lk));
    }
    std::vector<pss_cand> v;
    PSS_TRY(sift_across(*plan, *cfg, surv, &v, cfg->zmax ? &lk : nullptr));
    *n_out = (int64_t)v.size();
    if ((int64_t)v.size() > cap) return fail(PSS_ECAP, "pss_sift_in_batches: output capacity too small");
    if (!v.empty()) {
        if (!out) return fail(PSS_EINVAL, "pss_sift_in_batches: null out");
        memcpy(out, v.data(), v.size() * sizeof(pss_cand));
    }
    return PSS_OK;
}

pss_status pss_search_dm_batch(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data,
                               int data_on_device, const pss_search_cfg* cfg, int64_t dm_begin, int64_t dm_end,
                               pss_cand* out, int64_t cap, int64_t* n_out, void* stream) {
    if (!n_out) return fail(PSS_EINVAL, "pss_search_dm_batch: null n_out");
    *n_out = 0;
    if (ctx) PSS_CUDA(cudaSetDevice(ctx->device));
    if (!ctx) return fail(PSS_EINVAL, "null ctx");
    ctx->has_last = false;
    PSS_TRY(search_pipelined(ctx, plan, fil, data, data_on_device, cfg, dm_begin, dm_end, pick_stream(ctx, stream),
                             &ctx->last_cands));
    ctx->has_last = true;
    return take_cands(ctx->last_cands, out, cap, n_out);
}

pss_status pss_search_multi(pss_ctx* ctx, const pss_search_cfg* cfg, const pss_multi_file* files, int32_t nfiles,
                            int data_on_device, pss_cand* out, int64_t cap, int64_t* counts, int64_t* n_out,
                            void* stream) {
    if (!n_out || !counts) return fail(PSS_EINVAL, "pss_search_multi: null counts or n_out");
    *n_out = 0;
    if (!ctx) return fail(PSS_EINVAL, "null ctx");
    PSS_CUDA(cudaSetDevice(ctx->device));
    ctx->has_last = false;
    PSS_TRY(multi_search(ctx, cfg, files, nfiles, data_on_device, pick_stream(ctx, stream), &ctx->last_cands,
                         &ctx->last_counts));
    ctx->has_last = true;
    for (int32_t f = 0; f < nfiles; ++f) counts[f] = ctx->last_counts[f];
    return take_cands(ctx->last_cands, out, cap, n_out);
}

pss_status pss_search_multi_footprint(const pss_search_cfg* cfg, const pss_multi_file* files, int32_t nfiles,
                                      size_t* bytes) {
    if (!bytes || !cfg || !files || nfiles < 1) return fail(PSS_EINVAL, "pss_search_multi_footprint: null argument");
    *bytes = 0;
    std::vector<const Plan*> plans;
    std::vector<const pss_fil_desc*> fils;
    for (int32_t f = 0; f < nfiles; ++f) {
        if (!files[f].plan || !files[f].fil) return fail(PSS_EINVAL, "pss_search_multi_footprint: null plan or descriptor");
        if (files[f].plan->nsub > 0)
            return fail(PSS_EINVAL, "pss_search_multi_footprint: two-stage (subband) plans are not supported");
        PSS_TRY(validate_search(files[f].plan, files[f].fil, cfg));
        plans.push_back(files[f].plan);
        fils.push_back(files[f].fil);
    }
    *bytes = multi_footprint(plans, fils, cfg);
    return PSS_OK;
}

pss_status pss_ctx_take_cands(pss_ctx* ctx, pss_cand* out, int64_t cap, int64_t* n_out) {
    if (!ctx || !n_out) return fail(PSS_EINVAL, "pss_ctx_take_cands: null argument");
    *n_out = 0;
    if (!ctx->has_last) return fail(PSS_EINVAL, "pss_ctx_take_cands: the context holds no search result");
    return take_cands(ctx->last_cands, out, cap, n_out);
}

}  // extern "C"

namespace pss {
namespace {
__global__ void k_response(const double* q, const double* z, int64_t n, double* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const cplx r = rho_resp(q[i], z[i]);
    out[2 * i] = r.re;
    out[2 * i + 1] = r.im;
}
}  // namespace
}  // namespace pss

extern "C" pss_status pss_response(pss_ctx* ctx, const double* q, const double* z, int64_t n, double* out) {
    if (!ctx || (n > 0 && (!q || !z || !out)) || n < 0) return fail(PSS_EINVAL, "pss_response: bad arguments");
    if (n == 0) return PSS_OK;
    PSS_CUDA(cudaSetDevice(ctx->device));
    double* d = nullptr;
    PSS_CUDA(cudaMalloc(&d, (size_t)n * 4 * sizeof(double)));
    cudaStream_t s = ctx->stream;
    cudaError_t e = cudaMemcpyAsync(d, q, n * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + n, z, n * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_response<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(d, d + n, n, d + 2 * n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + 2 * n, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "pss_response");
    return PSS_OK;
}

// ---- candidate refinement --------------------------------------------------

namespace pss {
namespace {

const double K_DISP_REFINE = 4.148808e3;  // s MHz^2 pc^-1 cm^3

pss_status refine_prepare(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data, int on_dev,
                          const pss_search_cfg* cfg, int32_t stage, cudaStream_t s) {
    if (stage < 0 || stage >= (int)plan->stages.size()) return fail(PSS_EINVAL, "pss_refine_prepare: bad stage");
    const StageInfo& st = plan->stages[stage];
    const int64_t nfft = st.nfft, M = nfft / 2;
    // whitening gains of every trial of the stage (also stages the input)
    const int64_t nblocks = M / cfg->whiten_block;
    PSS_TRY(ctx->refine_gains.ensure((size_t)st.n_dm * nblocks * sizeof(float)));
    Outputs o;
    o.gains = (float*)ctx->refine_gains.p;
    PSS_TRY(run_path(ctx, plan, fil, data, on_dev, cfg, st.first, st.first + st.n_dm, MODE_GAINS, o, s, 0));
    // per-channel series (channel-major copy already staged by run_path) and spectra
    const std::vector<int32_t> keep = kept_channels(fil);
    const int32_t ck = (int32_t)keep.size();
    const int64_t pitch = xcm_pitch(*plan, fil);
    PSS_TRY(ctx->series.ensure((size_t)ck * nfft * 4));
    PSS_TRY(ctx->sums.ensure((size_t)ck * 8));
    PSS_TRY(ctx->fftA.ensure((size_t)ck * M * 8));
    PSS_TRY(ctx->fftB.ensure((size_t)ck * M * 8));
    PSS_TRY(ctx->chan_spec.ensure((size_t)ck * M * 8));
    PSS_CUDA(cudaMemsetAsync(ctx->sums.p, 0, (size_t)ck * 8, s));
    PSS_CUDA(launch_chan_series((const uint8_t*)ctx->xcm.p, pitch, ck, st.nv, st.ds, (float*)ctx->series.p, nfft,
                                (unsigned long long*)ctx->sums.p, s));
    FftArgs fa{};
    fa.series = (const float*)ctx->series.p;
    fa.series_stride = nfft;
    fa.sums = (const unsigned long long*)ctx->sums.p;
    fa.nv = st.nv;
    fa.nfft = nfft;
    fa.nb = ck;
    fa.bufA = (float2*)ctx->fftA.p;
    fa.bufB = (float2*)ctx->fftB.p;
    fa.spec_out = (float2*)ctx->chan_spec.p;
    fa.spec_stride = M;
    fa.whiten_block = cfg->whiten_block;
    fa.tw = (const float2*)ctx->twid.p;
    fa.twM = ctx->twid_n;
    fa.fft_variant = 0;
    PSS_TRY(ensure_passtw(ctx, M, 0, s));
    set_passtw(ctx, &fa);
    fa.whiten = 0;
    fa.gains_out = nullptr;
    fa.gains_stride = 0;
    PSS_CUDA(launch_fft_whiten(fa, s, ctx));
    // delay per unit DM of each kept channel, relative to the top channel
    double fmax = -1e300;
    for (double f : plan->freqs) fmax = std::max(fmax, f);
    std::vector<double> dt(ck);
    for (int32_t r = 0; r < ck; ++r) {
        const double f = plan->freqs[keep[r]];
        dt[r] = K_DISP_REFINE * (1.0 / (f * f) - 1.0 / (fmax * fmax));
    }
    PSS_TRY(ctx->refine_dtau.ensure((size_t)ck * sizeof(double)));
    PSS_CUDA(cudaMemcpyAsync(ctx->refine_dtau.p, dt.data(), ck * sizeof(double), cudaMemcpyHostToDevice, s));
    PSS_CUDA(cudaStreamSynchronize(s));
    ctx->refine_plan = plan;
    ctx->refine_stage = stage;
    ctx->refine_ck = ck;
    ctx->refine_nfft = nfft;
    ctx->refine_first = st.first;
    ctx->refine_ntrials = st.n_dm;
    ctx->refine_nblocks = nblocks;
    ctx->refine_extra = cfg->halfwidth_extra;
    ctx->refine_block = cfg->whiten_block;
    ctx->refine_T = (double)(nfft * (int64_t)st.ds) * plan->tsamp;
    return PSS_OK;
}

pss_status refine_eval(pss_ctx* ctx, const pss_plan* plan, const pss_refine_point* pts, int64_t n, double* power,
                       double* grad, cudaStream_t s) {
    if (ctx->refine_plan != plan || ctx->refine_stage < 0)
        return fail(PSS_EINVAL, "pss_refine_eval: call pss_refine_prepare for this plan first");
    std::vector<RefinePt> hp((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t t = (int64_t)pts[i].dm_idx - ctx->refine_first;
        if (t < 0 || t >= ctx->refine_ntrials)
            return fail(PSS_EINVAL, "pss_refine_eval: point outside the prepared stage");
        if (pts[i].numharm < 1 || pts[i].numharm > 32) return fail(PSS_EINVAL, "pss_refine_eval: bad numharm");
        if (!(pts[i].r >= 0.0) || !(pts[i].r * pts[i].numharm < ctx->refine_nfft / 2))
            return fail(PSS_EINVAL, "pss_refine_eval: r outside the spectrum");
        if ((int)ceil(fabs(pts[i].z * pts[i].numharm) / 2.0) + ctx->refine_extra > refine_max_taps() / 2)
            return fail(PSS_EINVAL, "pss_refine_eval: |z| too large");
        hp[(size_t)i] = RefinePt{(int32_t)t, pts[i].numharm, pts[i].dm, pts[i].r, pts[i].z};
    }
    if (n == 0) return PSS_OK;
    PSS_TRY(ctx->refine_pts.ensure((size_t)n * sizeof(RefinePt)));
    PSS_TRY(ctx->refine_out.ensure((size_t)n * 4 * sizeof(double)));
    PSS_CUDA(cudaMemcpyAsync(ctx->refine_pts.p, hp.data(), n * sizeof(RefinePt), cudaMemcpyHostToDevice, s));
    RefineArgs a;
    a.pts = (const RefinePt*)ctx->refine_pts.p;
    a.chan_spec = (const float2*)ctx->chan_spec.p;
    a.dtau = (const double*)ctx->refine_dtau.p;
    a.gains = (const float*)ctx->refine_gains.p;
    a.nfft = ctx->refine_nfft;
    a.ck = ctx->refine_ck;
    a.extra = ctx->refine_extra;
    a.whiten_block = ctx->refine_block;
    a.nblocks = ctx->refine_nblocks;
    a.T = ctx->refine_T;
    a.power = (double*)ctx->refine_out.p;
    a.grad = (double*)ctx->refine_out.p + n;
    PSS_CUDA(launch_refine_eval(a, n, s));
    PSS_CUDA(cudaMemcpyAsync(power, a.power, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (grad) PSS_CUDA(cudaMemcpyAsync(grad, a.grad, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
    PSS_CUDA(cudaStreamSynchronize(s));
    return PSS_OK;
}

}  // namespace
}  // namespace pss

extern "C" pss_status pss_refine_prepare(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data,
                                         int data_on_device, const pss_search_cfg* cfg, int32_t stage, void* stream) {
    PSS_TRY(check_common(ctx, plan, fil, data, 0, 0));
    PSS_TRY(check_cfg(cfg, *plan));
    PSS_CUDA(cudaSetDevice(ctx->device));
    return refine_prepare(ctx, plan, fil, data, data_on_device, cfg, stage, pick_stream(ctx, stream));
}

extern "C" pss_status pss_refine_eval(pss_ctx* ctx, const pss_plan* plan, const pss_refine_point* pts, int64_t n,
                                      double* power, double* grad, void* stream) {
    if (!ctx || !plan || (n > 0 && (!pts || !power)) || n < 0) return fail(PSS_EINVAL, "pss_refine_eval: bad arguments");
    PSS_CUDA(cudaSetDevice(ctx->device));
    return refine_eval(ctx, plan, pts, n, power, grad, pick_stream(ctx, stream));
}

extern "C" pss_status pss_refine_candidates(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil,
                                            const void* data, int data_on_device, const pss_search_cfg* cfg,
                                            pss_cand* inout, int64_t n, int32_t iters, double lr, void* stream) {
    PSS_TRY(check_common(ctx, plan, fil, data, 0, 0));
    PSS_TRY(check_cfg(cfg, *plan));
    if (n < 0 || (n > 0 && !inout) || iters < 0 || !(lr > 0)) return fail(PSS_EINVAL, "pss_refine_candidates: bad arguments");
    PSS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = pick_stream(ctx, stream);
    for (int64_t i = 0; i < n; ++i)
        if (inout[i].dm_idx < 0 || inout[i].dm_idx >= plan->ndm())
            return fail(PSS_EINVAL, "pss_refine_candidates: dm_idx outside the plan");
    const double dzc = cfg->zmax ? cfg->dz : 0.0;  // z moves only in an acceleration search
    for (size_t stg = 0; stg < plan->stages.size(); ++stg) {
        std::vector<int64_t> idx;
        for (int64_t i = 0; i < n; ++i)
            if (plan->stage_of[inout[i].dm_idx] == (int32_t)stg) idx.push_back(i);
        if (idx.empty()) continue;
        PSS_TRY(refine_prepare(ctx, plan, fil, data, data_on_device, cfg, (int32_t)stg, s));
        const double dm_cell = plan->stages[stg].dm_step > 0 ? plan->stages[stg].dm_step : 1.0;
        const size_t m = idx.size();
        // Adam on cell-normalised coordinates u = (DM / dm_step, r, z / dz)
        std::vector<pss_refine_point> cur(m), best(m);
        std::vector<double> bestP(m, -1.0), P(m), G(3 * m), mom(3 * m, 0.0), vel(3 * m, 0.0);
        std::vector<double> u0(3 * m);
        for (size_t q = 0; q < m; ++q) {
            const pss_cand& c = inout[idx[q]];
            cur[q] = pss_refine_point{c.dm_idx, c.numharm, c.dm, c.r, c.z};
            u0[3 * q] = c.dm / dm_cell;
            u0[3 * q + 1] = c.r;
            u0[3 * q + 2] = dzc > 0 ? c.z / dzc : 0.0;
        }
        const double b1 = 0.9, b2 = 0.999, eps = 1e-12;
        for (int it = 0; it <= iters; ++it) {
            PSS_TRY(refine_eval(ctx, plan, cur.data(), (int64_t)m, P.data(), G.data(), s));
            for (size_t q = 0; q < m; ++q) {
                if (P[q] > bestP[q]) {
                    bestP[q] = P[q];
                    best[q] = cur[q];
                }
            }
            if (it == iters) break;
            for (size_t q = 0; q < m; ++q) {
                const double gu[3] = {G[3 * q] * dm_cell, G[3 * q + 1], dzc > 0 ? G[3 * q + 2] * dzc : 0.0};
                double u[3] = {cur[q].dm / dm_cell, cur[q].r, dzc > 0 ? cur[q].z / dzc : 0.0};
                for (int d = 0; d < 3; ++d) {
                    double& mo = mom[3 * q + d];
                    double& ve = vel[3 * q + d];
                    mo = b1 * mo + (1 - b1) * gu[d];
                    ve = b2 * ve + (1 - b2) * gu[d] * gu[d];
                    const double mh = mo / (1 - pow(b1, it + 1)), vh = ve / (1 - pow(b2, it + 1));
                    u[d] += lr * mh / (sqrt(vh) + eps);  // ascent
                    // stay within two cells of the detection
                    u[d] = std::min(std::max(u[d], u0[3 * q + d] - 2.0), u0[3 * q + d] + 2.0);
                }
                cur[q].dm = std::max(0.0, u[0] * dm_cell);
                cur[q].r = std::max(0.5, u[1]);
                cur[q].z = dzc > 0 ? u[2] * dzc : 0.0;
            }
        }
        for (size_t q = 0; q < m; ++q) {
            pss_cand& c = inout[idx[q]];
            c.dm = best[q].dm;
            c.r = best[q].r;
            c.z = best[q].z;
            c.f_hz = best[q].r / ctx->refine_T;
            c.power = (float)bestP[q];
            c.sigma = sigma_of_power(c.numharm, bestP[q]);
        }
    }
    return PSS_OK;
}

// ---- prepared, graph-captured search of one file shape ---------------------

struct pss_batch {
    pss_ctx* ctx = nullptr;
    pss::Plan plan;
    pss_fil_desc fil{};
    std::vector<uint8_t> mask;
    pss_search_cfg cfg{};
    pss::PathSetup P;
    std::vector<pss_cand> last;  // sifted candidates of the last run
    bool has_last = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t footprint = 0;
};

namespace pss {
namespace {

size_t ctx_bytes(const pss_ctx* c) {
    const DevBuf* bufs[] = {&c->fil_dev, &c->xcm, &c->delays_dev, &c->subu, &c->bx, &c->series, &c->sums, &c->fftA,
                            &c->fftB, &c->spec, &c->plane, &c->cands, &c->counter, &c->taps, &c->ftaps, &c->tapinfo,
                            &c->errflag, &c->twid, &c->mf_fil, &c->mf_xcm, &c->mf_work};
    size_t t = 0;
    for (const DevBuf* b : bufs) t += b->bytes;
    for (const auto& p : c->passtw) t += p.buf.bytes;
    return t;
}

void batch_release_graph(pss_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// ---- autotuner ----------------------------------------------------------------
//
// A prepared batch picks its launch shapes by timing them: on the first
// min(ndm, 256) trials of its file shape (the input in ctx->fil_dev), each
// choice is tried in turn (FFT pass split, harmonic-sum points per lane,
// dedispersion chunk budget, whitening form), each candidate run once to
// warm and once with the stage it changes timed by CUDA events, and the
// fastest kept.  The result is remembered per shape for the life of the
// process, so every batch of a shape (and so every file of that shape in a
// server) runs the same kernels.  PSS_AUTOTUNE=0 disables it; PSS_TUNE pins
// the choices.

std::string tune_key(const Plan& plan, const pss_fil_desc* f, const pss_search_cfg* c) {
    std::string k;
    char buf[256];
    snprintf(buf, sizeof buf, "%d/%d/%lld/%.17g/%.17g/%.17g/%d|", f->nchan, f->nbits, (long long)f->nsamp,
             f->tsamp_s, f->fch0_mhz, f->foff_mhz, f->layout);
    k += buf;
    for (int i = 0; i < f->nchan; ++i) k += (f->chan_mask && !f->chan_mask[i]) ? '0' : '1';
    snprintf(buf, sizeof buf, "|sub%d,%d", plan.nsub, plan.sub_group);
    k += buf;
    for (const auto& st : plan.stages) {
        snprintf(buf, sizeof buf, "|%.17g,%.17g,%d,%d", st.dm_lo, st.dm_step, st.n_dm, st.ds);
        k += buf;
    }
    snprintf(buf, sizeof buf, "|%d,%d,%.17g,%.17g,%.17g,%d,%d,%d", c->zmax, c->numharm, c->dz, c->sigma_thr,
             c->f_lo_hz, c->whiten_block, c->halfwidth_extra, c->min_dm_hits);
    k += buf;
    return k;
}

std::mutex g_tune_mu;
std::map<std::string, Tune> g_tuned;

pss_status autotune(pss_ctx* ctx, const Plan& plan, const pss_fil_desc* fil, const pss_search_cfg* cfg) {
    // PSS_TUNE="fft,harm,dedisp,whiten" pins the launch shapes instead (not remembered)
    // (the fft split applies to every stage's size that has such a split, the even split elsewhere)
    if (const char* pin = getenv("PSS_TUNE")) {
        Tune t;
        int split = 0;
        const int got = sscanf(pin, "%d,%d,%d,%d,%d,%d", &split, &t.harm_run, &t.dedisp_kb, &t.whiten_form,
                               &t.fused, &t.plane_form);
        if (got < 4)
            return fail(PSS_EINVAL, "PSS_TUNE must be 4 to 6 integers: fft split, harm run, dedisp KiB, whiten form"
                                    "[, fused[, plane form]]");
        if ((t.fused != 0 && t.fused != 1) || (t.plane_form != 0 && t.plane_form != 1))
            return fail(PSS_EINVAL, "PSS_TUNE value out of range");
        int rad[4];
        if (split < 0 || fft_pass_plan(plan.stages[0].nfft / 2, split, rad) == 0 ||
            (t.harm_run != 8 && t.harm_run != 16) || t.dedisp_kb < 16 || t.dedisp_kb > 200 || t.whiten_form < -1 ||
            t.whiten_form > 2)
            return fail(PSS_EINVAL, "PSS_TUNE value out of range");
        for (const auto& st : plan.stages) {
            const int64_t M = st.nfft / 2;
            int L = 0;
            while (L < 31 && (int64_t(1) << L) < M) ++L;
            t.fft_split[L] = (int8_t)(fft_pass_plan(M, split, rad) > 0 ? split : 0);
        }
        ctx->tune = t;
        return PSS_OK;
    }
    const char* env = getenv("PSS_AUTOTUNE");
    if (env && env[0] == '0') return PSS_OK;
    const std::string key = tune_key(plan, fil, cfg);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            ctx->tune = it->second;
            return PSS_OK;
        }
    }
    cudaStream_t s = ctx->stream;
    const pss_plan* pp = static_cast<const pss_plan*>(&plan);
    // trials the choices are timed on: the first min(n, 256) of the plan, or of the stage being tuned
    int64_t tb = 0, te = std::min<int64_t>(plan.ndm(), 256);
    // time of profiler stage `stage` (1 dedisperse, 2 FFT, 3 whiten, 5 harmonic sum) over one
    // warm pass; the kernels of the other stages do not change with the choice being tuned
    auto measure = [&](unsigned stages, float* ms) -> pss_status {
        PathSetup T;
        PSS_TRY(setup_path(ctx, pp, fil, cfg, tb, te, MODE_SEARCH, s, kBatchInitialCap, &T));
        const uint8_t* src = (const uint8_t*)ctx->fil_dev.p;
        PSS_TRY(enqueue_path(ctx, pp, fil, src, cfg, tb, T, MODE_SEARCH, Outputs(), s));
        PSS_TRY(pss_ctx_profile(ctx, 1));
        PSS_TRY(enqueue_path(ctx, pp, fil, src, cfg, tb, T, MODE_SEARCH, Outputs(), s));
        double st_ms[PSS_NPROF_STAGES];
        int64_t n[PSS_NPROF_STAGES];
        pss_status r = pss_ctx_profile_read(ctx, st_ms, n);
        pss_ctx_profile(ctx, 0);
        PSS_TRY(r);
        *ms = 0.f;
        for (int i = 0; i < PSS_NPROF_STAGES; ++i)
            if (stages & (1u << i)) *ms += (float)st_ms[i];
        return check_errflag(ctx, s);
    };
    auto sweep = [&](auto* field, const std::vector<int>& cands, unsigned stage, const char* what) -> pss_status {
        int best = *field;
        float best_ms = 1e30f;
        for (int v : cands) {
            *field = v;
            float ms = 0.f;
            PSS_TRY(measure(stage, &ms));
            if (getenv("PSS_TIMING")) fprintf(stderr, "[pss] tune %-10s %5d: %8.3f ms\n", what, v, ms);
            if (ms < best_ms) {
                best_ms = ms;
                best = v;
            }
        }
        *field = best;
        return PSS_OK;
    };
    pss_status st = PSS_OK;
    {
        // stage bits of the profiler: 1 dedisperse, 2 FFT (and the fused kernel), 3 whiten, 4 plane, 5 harmonic sum
        const bool fusable = cfg->zmax == 0 && plan.stages.size() == 1 && plan.stages[0].nfft == (int64_t(1) << 18) &&
                             cfg->whiten_block == 1024 && cfg->halfwidth_extra == 16 && spec_cluster_usable();
        if (fusable) st = sweep(&ctx->tune.fused, {1, 0}, (1u << 2) | (1u << 3) | (1u << 4), "fused");
        else ctx->tune.fused = 0;
        if (st == PSS_OK && !ctx->tune.fused) {
            // FFT pass splits of every transform size of the plan, each timed on the first
            // trials of the first stage of that size
            for (size_t si = 0; si < plan.stages.size() && st == PSS_OK; ++si) {
                const auto& sg = plan.stages[si];
                const int64_t M = sg.nfft / 2;
                bool seen = sg.n_dm == 0;
                for (size_t sj = 0; sj < si && !seen; ++sj) seen = plan.stages[sj].n_dm > 0 && plan.stages[sj].nfft == sg.nfft;
                if (seen) continue;
                std::vector<int> fv;
                int rad[4];
                for (int v = 0; v < 6 && fft_pass_plan(M, v, rad) > 0; ++v) fv.push_back(v);
                int L = 0;
                while (L < 31 && (int64_t(1) << L) < M) ++L;
                tb = sg.first;
                te = sg.first + std::min<int64_t>(sg.n_dm, 256);
                if (fv.size() > 1) st = sweep(&ctx->tune.fft_split[L], fv, 1u << 2, "fft split");
            }
            tb = 0;
            te = std::min<int64_t>(plan.ndm(), 256);
            if (st == PSS_OK) st = sweep(&ctx->tune.whiten_form, {0, 1, 2}, 1u << 3, "whiten");
        } else {
            ctx->tune.whiten_form = 0;  // not used by the fused kernel
        }
        if (st == PSS_OK && cfg->zmax > 0 && plane_fft_usable(cfg->zmax, cfg->halfwidth_extra, plan.stages[0].nfft / 2))
            st = sweep(&ctx->tune.plane_form, {1, 0}, 1u << 4, "plane form");
        if (st == PSS_OK) st = sweep(&ctx->tune.harm_run, {8, 16}, 1u << 5, "harm run");
        if (st == PSS_OK) st = sweep(&ctx->tune.dedisp_kb, {96, 64}, 1u << 1, "dedisp kb");
    }
    if (st != PSS_OK) {
        ctx->tune = Tune();
        return st;
    }
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tuned.emplace(key, ctx->tune);
    return PSS_OK;
}

// (Re)build the set-up for the full DM range with candidate capacity `cap`
// and capture the kernel sequence into a graph (input: ctx->fil_dev).
pss_status batch_build(pss_batch* b, int64_t cap) {
    pss_ctx* ctx = b->ctx;
    cudaStream_t s = ctx->stream;
    batch_release_graph(b);
    const int64_t n = b->plan.ndm();
    PSS_TRY(setup_path(ctx, static_cast<const pss_plan*>(&b->plan), &b->fil, &b->cfg, 0, n, MODE_SEARCH, s, cap,
                       &b->P, pipeline_batch(n)));
    PSS_TRY(ctx->fil_dev.ensure((size_t)file_bytes(&b->fil)));
    PSS_TRY(ensure_snapshots(ctx, (int)b->P.batches.size()));
    // one eager pass sets every kernel attribute before capture
    PSS_TRY(enqueue_path(ctx, static_cast<const pss_plan*>(&b->plan), &b->fil, (const uint8_t*)ctx->fil_dev.p,
                         &b->cfg, 0, b->P, MODE_SEARCH, Outputs(), s, true));
    PSS_CUDA(cudaStreamSynchronize(s));
    // relaxed: the launchers call cudaFuncSetAttribute, which is not a stream operation
    PSS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    pss_status st = enqueue_path(ctx, static_cast<const pss_plan*>(&b->plan), &b->fil, (const uint8_t*)ctx->fil_dev.p,
                                 &b->cfg, 0, b->P, MODE_SEARCH, Outputs(), s, true);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != PSS_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
        batch_release_graph(b);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    b->footprint = ctx_bytes(ctx);
    return PSS_OK;
}

}  // namespace
}  // namespace pss

extern "C" pss_status pss_batch_create(int device, const pss_plan* plan, const pss_fil_desc* fil,
                                       const pss_search_cfg* cfg, pss_batch** out) {
    if (!out || !plan || !fil || !cfg) return fail(PSS_EINVAL, "pss_batch_create: null argument");
    *out = nullptr;
    PSS_TRY(check_common(reinterpret_cast<pss_ctx*>(1), plan, fil, fil, 0, 0));
    PSS_TRY(check_cfg(cfg, *plan));
    pss_batch* b = new pss_batch();
    pss_status st = pss_ctx_create(device, &b->ctx);
    if (st != PSS_OK) {
        delete b;
        return st;
    }
    b->plan = *plan;
    b->fil = *fil;
    if (fil->chan_mask) {
        b->mask.assign(fil->chan_mask, fil->chan_mask + fil->nchan);
        b->fil.chan_mask = b->mask.data();
    }
    b->cfg = *cfg;
    st = b->ctx->fil_dev.ensure((size_t)file_bytes(&b->fil));
    if (st == PSS_OK) {
        // tune on a constant file (the kernels' work does not depend on the values)
        cudaError_t e = cudaMemsetAsync(b->ctx->fil_dev.p, 0x80, (size_t)file_bytes(&b->fil), b->ctx->stream);
        st = e == cudaSuccess ? autotune(b->ctx, b->plan, &b->fil, &b->cfg) : cuda_fail(e, "cudaMemsetAsync");
    }
    if (st == PSS_OK) st = batch_build(b, kBatchInitialCap);
    if (st != PSS_OK) {
        const std::string msg = pss_last_error();
        pss_batch_free(b);
        return fail(st, msg);
    }
    *out = b;
    return PSS_OK;
}

namespace pss {

// Device bytes a pss_batch of this shape will hold (the DevBuf sizes
// setup_path and the templates ask for, with DevBuf's slack), computed on
// the host without touching the device: the server admits files by it.
pss_status validate_search(const pss_plan* plan, const pss_fil_desc* fil, const pss_search_cfg* cfg) {
    PSS_TRY(check_common(reinterpret_cast<pss_ctx*>(1), plan, fil, fil, 0, 0));
    return check_cfg(cfg, *plan);
}

size_t search_footprint(const Plan& plan, const pss_fil_desc* fil, const pss_search_cfg* cfg, int64_t dev_cap) {
    auto buf = [](size_t want) { return want ? want + want / 8 + 256 : (size_t)0; };
    const std::vector<int32_t> keep = kept_channels(fil);
    const int64_t ck = (int64_t)keep.size();
    const int64_t pitch = xcm_pitch(plan, fil);
    const int nz = nz_of(cfg);
    size_t tables = (size_t)(ck + plan.ndm() * ck);
    if (plan.nsub > 0) {
        const size_t ng = plan.grp_first.size();
        tables = std::max(tables, (size_t)ck + ng * ck + (size_t)plan.ndm() * plan.nsub + 2 * ng + 2 * plan.nsub + 16);
    }
    size_t t = buf((size_t)file_bytes(fil)) + buf((size_t)ck * pitch + 64) + buf(tables * sizeof(int32_t)) +
               buf(sizeof(int)) + buf((size_t)dev_cap * sizeof(pss_raw_cand)) + buf(sizeof(unsigned long long));
    int64_t nfft_max = 0, total_taps = 0;
    size_t need_series = 0, need_fft = 0, need_sums = 0, need_plane = 0, subu = 0, bx = 0;
    Tune bx_tune;  // the boxcar-table threshold a new context takes (environment included)
    if (const char* f = getenv("PSS_DEDISP_BX_MIN")) bx_tune.bx_min = std::max(0, atoi(f));
    std::vector<int64_t> sizes;
    for (const auto& st : plan.stages) {
        nfft_max = std::max<int64_t>(nfft_max, st.nfft);
        if (st.n_dm <= 0) continue;
        if (plan.nsub == 0 && bx_use(bx_tune, st.ds) && ck <= 65535) bx = std::max(bx, bx_table_bytes((int32_t)ck, plan.nsamp, st.ds));
        if (std::find(sizes.begin(), sizes.end(), st.nfft) == sizes.end()) {
            sizes.push_back(st.nfft);
            t += buf((size_t)(st.nfft / 2) * sizeof(float2));  // inter-pass twiddles (at most M entries)
        }
        const int64_t B = batch_trials(st.nfft, nz, MODE_SEARCH, st.n_dm);
        if (plan.nsub > 0) {
            // stage-1 rows: groups touched by a batch x subbands x (N_v ds + largest D, padded)
            const int64_t ngb = (B + plan.sub_group - 1) / plan.sub_group + 1;
            subu = std::max(subu, (size_t)plan.nsub * ngb * ((fil->nsamp + 3) & ~int64_t(3)) * 4 +
                                      subsum_slack_bytes((int32_t)plan.max_delay));
        }
        need_series = std::max(need_series, (size_t)B * st.nfft * 4);
        need_sums = std::max(need_sums, (size_t)B * 8);
        need_fft = std::max(need_fft, (size_t)B * (st.nfft / 2) * 8);
        need_plane = std::max(need_plane, (size_t)B * nz * st.nfft * 4);
    }
    for (int j = 0; j < nz; ++j) {
        const double z = cfg->zmax ? -(double)cfg->zmax + (double)j * cfg->dz : 0.0;
        total_taps += 4 * ((int64_t)ceil(fabs(z) / 2.0) + cfg->halfwidth_extra);
    }
    if (plane_fft_usable(cfg->zmax, cfg->halfwidth_extra, PLANE_FFT_L))
        t += buf((size_t)nz * 2 * PLANE_FFT_L * sizeof(float2));
    t += buf((size_t)nfft_max * sizeof(float2)) + buf(need_series) + buf(need_sums) + 3 * buf(need_fft) +
         buf(need_plane) + buf((size_t)total_taps * sizeof(float2)) + buf((size_t)5 * nz * sizeof(int32_t)) +
         buf(subu) + buf(bx);
    return t;
}

}  // namespace pss

extern "C" pss_status pss_search_footprint(const pss_plan* plan, const pss_fil_desc* fil, const pss_search_cfg* cfg,
                                           size_t* bytes) {
    if (!bytes) return fail(PSS_EINVAL, "pss_search_footprint: null argument");
    PSS_TRY(validate_search(plan, fil, cfg));
    *bytes = search_footprint(*plan, fil, cfg, kBatchInitialCap);
    return PSS_OK;
}

extern "C" size_t pss_batch_footprint(const pss_batch* b) { return b ? b->footprint : 0; }

extern "C" pss_status pss_batch_tuning(const pss_batch* b, int32_t* fft_split, int32_t* harm_run, int32_t* dedisp_kb,
                                       int32_t* whiten_form, int32_t* fused) {
    if (!b) return fail(PSS_EINVAL, "pss_batch_tuning: null batch");
    if (fft_split) *fft_split = b->ctx->tune.split_for(b->plan.stages[0].nfft / 2);
    if (harm_run) *harm_run = b->ctx->tune.harm_run;
    if (dedisp_kb) *dedisp_kb = b->ctx->tune.dedisp_kb;
    if (whiten_form) *whiten_form = b->ctx->tune.whiten_form;
    if (fused) *fused = b->ctx->tune.fused;
    return PSS_OK;
}

namespace {
// log2 of an FFT's complex points M = nfft / 2 (nfft a power of two >= 128), or -1
int split_index(int64_t nfft) {
    if (nfft < 128 || (nfft & (nfft - 1)) != 0) return -1;
    int L = 0;
    while ((int64_t(1) << L) < nfft / 2) ++L;
    return L < 32 ? L : -1;
}
}  // namespace

extern "C" pss_status pss_fft_split_radices(int64_t nfft, int32_t split, int32_t* npass, int32_t* radices) {
    if (!npass || !radices) return fail(PSS_EINVAL, "pss_fft_split_radices: null argument");
    *npass = 0;
    if (split_index(nfft) < 0 || split < 0) return fail(PSS_EINVAL, "pss_fft_split_radices: bad nfft or split");
    int rad[4] = {0, 0, 0, 0};
    const int np = fft_pass_plan(nfft / 2, split, rad);
    if (np == 0) return fail(PSS_EINVAL, "pss_fft_split_radices: no such split for this size");
    for (int i = 0; i < 4; ++i) radices[i] = i < np ? rad[i] : 0;
    *npass = np;
    return PSS_OK;
}

extern "C" pss_status pss_ctx_set_fft_split(pss_ctx* ctx, int64_t nfft, int32_t split) {
    if (!ctx) return fail(PSS_EINVAL, "pss_ctx_set_fft_split: null ctx");
    const int L = split_index(nfft);
    int rad[4];
    if (L < 0 || split < 0 || split > 127 || fft_pass_plan(nfft / 2, split, rad) == 0)
        return fail(PSS_EINVAL, "pss_ctx_set_fft_split: no such split for this size");
    ctx->tune.fft_split[L] = (int8_t)split;
    return PSS_OK;
}

extern "C" pss_status pss_batch_fft_split(const pss_batch* b, int64_t nfft, int32_t* split) {
    if (!b || !split) return fail(PSS_EINVAL, "pss_batch_fft_split: null argument");
    const int L = split_index(nfft);
    if (L < 0) return fail(PSS_EINVAL, "pss_batch_fft_split: bad nfft");
    *split = b->ctx->tune.fft_split[L];
    return PSS_OK;
}

extern "C" pss_status pss_batch_run(pss_batch* b, const void* data, int data_on_device, pss_cand* out, int64_t cap,
                                    int64_t* n_out, double* gpu_ms) {
    if (!b || !data || !n_out) return fail(PSS_EINVAL, "pss_batch_run: null argument");
    *n_out = 0;
    pss_ctx* ctx = b->ctx;
    PSS_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const size_t nbytes = (size_t)file_bytes(&b->fil);
    b->has_last = false;
    b->last.clear();
    for (int attempt = 0; attempt < 2; ++attempt) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (gpu_ms) {
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, s);
        }
        PSS_CUDA(cudaMemcpyAsync(ctx->fil_dev.p, data, nbytes,
                                 data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        PSS_CUDA(cudaGraphLaunch(b->exec, s));
        if (gpu_ms) cudaEventRecord(e1, s);
        // the within-trial sift of each DM batch runs while the graph does the later ones
        std::vector<SiftItem> surv;
        SiftLinker lk;
        bool overflow = false;
        unsigned long long total = 0;
        PSS_TRY(drain_batches(ctx, static_cast<const pss_plan*>(&b->plan), &b->cfg, b->P.batches.size(),
                              b->P.dev_cap, &surv, &overflow, &total, &lk));
        PSS_CUDA(cudaStreamSynchronize(s));
        if (gpu_ms) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            *gpu_ms = ms;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
        PSS_TRY(check_errflag(ctx, s));
        if (!overflow) {
            PSS_TRY(sift_across(b->plan, b->cfg, surv, &b->last, b->cfg.zmax ? &lk : nullptr));
            b->has_last = true;
            return take_cands(b->last, out, cap, n_out);
        }
        // the candidate buffer overflowed: rebuild with room for all of them and redo
        if (attempt == 1) break;
        PSS_TRY(batch_build(b, (int64_t)total + 1024));
    }
    return fail(PSS_ECAP, "pss_batch_run: candidate buffer overflow persisted after resizing");
}

extern "C" pss_status pss_batch_take_cands(pss_batch* b, pss_cand* out, int64_t cap, int64_t* n_out) {
    if (!b || !n_out) return fail(PSS_EINVAL, "pss_batch_take_cands: null argument");
    *n_out = 0;
    if (!b->has_last) return fail(PSS_EINVAL, "pss_batch_take_cands: the batch holds no search result");
    return take_cands(b->last, out, cap, n_out);
}

extern "C" void pss_batch_free(pss_batch* b) {
    if (!b) return;
    if (b->ctx) {
        cudaSetDevice(b->ctx->device);
        batch_release_graph(b);
        pss_ctx_destroy(b->ctx);
    }
    delete b;
}

namespace pss {
size_t ctx_device_bytes(const pss_ctx* c) { return ctx_bytes(c); }
}  // namespace pss
