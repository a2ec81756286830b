// Internal declarations shared by the libpss translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <memory>
#include <string>
#include <thread>
#include <set>
#include <vector>

#include "../../include/pss.h"

namespace pss {

// ---- errors ---------------------------------------------------------------
void set_error(const std::string& msg);
pss_status fail(pss_status st, const std::string& msg);
pss_status cuda_fail(cudaError_t e, const char* what);

#define PSS_CUDA(call)                                          \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return pss::cuda_fail(_e, #call); \
    } while (0)

#define PSS_TRY(call)                      \
    do {                                   \
        pss_status _s = (call);            \
        if (_s != PSS_OK) return _s;       \
    } while (0)

// ---- plan -----------------------------------------------------------------
struct StageInfo {
    double dm_lo, dm_step;
    int32_t n_dm, ds;
    int64_t first;  // index of the stage's first trial
    int64_t nv, nfft;
};

struct Plan {
    int32_t nchan = 0;
    int64_t nsamp = 0;
    double tsamp = 0, fch0 = 0, foff = 0;
    std::vector<double> freqs;
    std::vector<StageInfo> stages;
    std::vector<double> dms;
    std::vector<int32_t> stage_of;
    std::vector<int32_t> delays;  // [ndm][nchan]
    int64_t max_delay = 0;        // D (or D' of the two-stage scheme)
    uint64_t id = 0;              // unique per plan built in this process
    // two-stage (subband) scheme; nsub == 0: exact shift-and-sum
    int32_t nsub = 0, sub_group = 0, sub_S = 0;
    std::vector<double> fsub;        // [nsub] reference frequency of each subband
    std::vector<int64_t> grp_first;  // [ngroups] first trial of each group
    std::vector<int32_t> grp_n;      // [ngroups] trials in each group
    std::vector<double> grp_dm;      // [ngroups] nominal DM
    std::vector<int32_t> grp_of;     // [ndm] group of each trial
    std::vector<int32_t> sub_e;      // [ngroups][nchan] within-subband delays at the nominal DM
    std::vector<int32_t> sub_D;      // [ndm][nsub] subband delays
    int64_t ndm() const { return (int64_t)dms.size(); }
    double t_span(int64_t dm) const {
        const StageInfo& s = stages[stage_of[dm]];
        return (double)(s.nfft * (int64_t)s.ds) * tsamp;
    }
};

pss_status build_plan(const pss_fil_desc* fil, const pss_dd_stage* st, int nst, Plan* out);
// The two-stage tables on top of a built plan; raises max_delay to D' and
// recomputes the stage lengths.
pss_status build_subband(Plan* P, int32_t nsub, int32_t group);

// ---- statistics (host) ----------------------------------------------------
double log_q(int n, double S);
double sigma_from_logp(double logp);
double sigma_of_power(int n, double S);
double power_threshold(int n, double sigma);

// ---- host parallel loop -----------------------------------------------------
// f(i) for i in [0, n) in chunks of `grain`, run by the calling thread and
// the workers of a process-wide pool (hardware_concurrency - 1 threads,
// started on first use).  Several callers (server slots) may run loops at
// once; each waits only for its own.
void parallel_for_fn(int64_t n, int64_t grain, const std::function<void(int64_t)>& f);
template <class F>
void parallel_for(int64_t n, int64_t grain, F&& f) {
    if (n <= grain) {
        for (int64_t i = 0; i < n; ++i) f(i);
        return;
    }
    const std::function<void(int64_t)> fn = std::forward<F>(f);
    parallel_for_fn(n, grain, fn);
}

// Stable counting sort of raw detections by DM index: returns the order
// and, for each DM present, [begin, end) into it.
void bucket_by_dm(const pss_raw_cand* raw, int64_t n, int64_t ndm, std::vector<int64_t>* order,
                  std::vector<std::pair<int64_t, int64_t>>* buckets);
// Sort raw detections by (dm_idx, numharm, j, h) in place.
void sort_raw(std::vector<pss_raw_cand>* v, int64_t ndm);

// Copy a kept candidate list to a caller's buffer (PSS_ECAP if it does not fit).
pss_status take_cands(const std::vector<pss_cand>& v, pss_cand* out, int64_t cap, int64_t* n_out);

// ---- sift (host) ----------------------------------------------------------
pss_status sift(const Plan& P, const pss_search_cfg& cfg, const pss_raw_cand* raw, int64_t n,
                std::vector<pss_cand>* out);
// The two halves of sift: survivors of the within-trial linkage (appended to
// *out; raw detections of one DM trial must all be in one call), then the
// across-trial linkage of all survivors.
struct SiftItem {
    int32_t dm_idx, n, h, j;
    float power;
    double r, z;
    double logp;     // log Q(n, S); NAN until evaluated
    double sigma;    // -Phi^-1(Q); < 0 until evaluated
    int64_t kr, kz;  // exact link coordinates: 64 r and 32 z / dz
};
pss_status sift_within(const Plan& P, const pss_search_cfg& cfg, const pss_raw_cand* raw, int64_t n,
                       std::vector<SiftItem>* out);
// Incremental single linkage of the survivors of 2-D planes (the links of
// sift_across, whose components do not depend on the order items arrive in):
// add() links the items [from, size) to those added before; groups() gives
// the components of all of them (members as item indices).
class SiftLinker {
  public:
    void add(const std::vector<SiftItem>& items, size_t from);
    void groups(std::vector<int>* start, std::vector<int>* members) const;
    size_t size() const { return cell_of_.size(); }

  private:
    struct LCell {
        int64_t cr, cz;
        int64_t r_lo, r_hi, z_lo, z_hi;
        std::vector<int> mem;
    };
    int find_cell(int64_t cr, int64_t cz) const;
    int root(int c) const;
    void grow();
    std::vector<LCell> cells_;
    std::vector<int> table_;   // open addressing: cell index or -1
    mutable std::vector<int> par_;
    std::vector<int> cell_of_;  // cell of each item
};
pss_status sift_across(const Plan& P, const pss_search_cfg& cfg, std::vector<SiftItem>& survivors,
                       std::vector<pss_cand>* out, const SiftLinker* linked = nullptr);

// ---- device workspace -----------------------------------------------------
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    pss_status ensure(size_t want);
    void release();
};

// Launch-shape choices the autotuner may change (pss_batch_create); the
// defaults are what untuned calls use.
struct Tune {
    // FFT pass split per transform size: fft_split[L] is the variant used for
    // M = 2^L complex points (0: the even split; see fft_pass_plan)
    int8_t fft_split[32] = {};
    int split_for(int64_t M) const {
        int L = 0;
        while (L < 31 && (int64_t(1) << L) < M) ++L;
        return fft_split[L];
    }
    int harm_run = 8;      // harmonic-sum points per lane
    int dedisp_kb = 96;    // dedispersion chunk staging budget
    int whiten_form = -1;  // whitening kernel form (-1: default, the warp pair per block)
    int fused = 0;         // zmax 0, nfft 2^18: cluster-fused FFT + whitening + plane (where the device allows)
    int plane_form = 1;    // overlap-save plane kernel form (1: radix 16-16-8, 0: radix 8-8-8-4)
    int bx_min = 8;        // rows with ds >= bx_min (and <= 256) dedisperse from the boxcar table (0: never)
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    DevBuf fil_dev;      // uploaded file bytes
    DevBuf xcm;          // channel-major uint8 [Ck][pitch]
    DevBuf delays_dev;   // int32 [ndm][Ck] (kept channels), or the two-stage tables
    DevBuf subu;         // int32 stage-1 subband sums of the two-stage scheme
    DevBuf sp_series;    // int32 dedispersed series of the single-pulse search
    DevBuf sp_mom;       // unsigned long long [2][B] moments
    DevBuf sp_ev;        // SpRaw detections
    DevBuf fold_buf;     // folding items and outputs
    DevBuf bx;           // uint16 boxcar table of the downsampled rows
    int bx_ds = 0;       // the ds the table holds for the current channel-major file (0: none)
    std::vector<int32_t> delays_host;  // what delays_dev holds (keep list + delays), empty if unknown
    uint64_t delays_gen = 0;           // bumped whenever delays_dev is rewritten
    std::shared_ptr<void> path_cache;  // last search set-up (api.cu), valid while delays_gen matches
    DevBuf series;       // float [B][nfft]
    DevBuf sums;         // unsigned long long [B]
    DevBuf fftA, fftB;   // float2 [B][M]
    DevBuf spec;         // float2 [B][M]  whitened spectrum
    DevBuf plane;        // float [B][nz][nfft]
    DevBuf cands;        // pss_raw_cand [cap]
    DevBuf counter;      // unsigned long long
    DevBuf taps;         // float2 templates
    DevBuf ftaps;        // float2 [nz][2][L] template spectra (overlap-save plane)
    DevBuf tapinfo;      // per row tap info
    DevBuf errflag;      // int: a kernel's bounded wait expired
    DevBuf twid;         // float2 twiddle table exp(-2 pi i t / twid_n)
    int64_t twid_n = 0;
    // inter-pass twiddle tables of each FFT size in use (later passes, laid out like their data)
    struct PassTw {
        int64_t M = 0, twM = 0;
        int variant = 0;
        DevBuf buf;
        int64_t off[4] = {0, 0, 0, 0};
    };
    std::vector<PassTw> passtw;
    // refinement state (pss_refine_prepare)
    DevBuf chan_spec, refine_gains, refine_dtau, refine_pts, refine_out;
    const void* refine_plan = nullptr;
    int32_t refine_stage = -1, refine_ck = 0, refine_extra = 16, refine_block = 1024;
    int64_t refine_nfft = 0, refine_first = 0, refine_ntrials = 0, refine_nblocks = 0;
    double refine_T = 0.0;
    void* host_pinned = nullptr;
    size_t host_pinned_bytes = 0;
    // (zmax, extra, dz) of the templates currently in `taps`
    int32_t tap_zmax = -1, tap_extra = -1;
    double tap_dz = 0.0;
    bool ftap_ok = false;  // ftaps hold the spectra of the current templates
    Tune tune;             // launch shapes (set by the autotuner of a prepared batch)
    // pipelined search: a second stream for candidate downloads, one event and
    // one pinned detection-count slot per DM batch
    cudaStream_t stream2 = nullptr;
    std::vector<cudaEvent_t> batch_ev;
    unsigned long long* batch_cnt = nullptr;  // pinned host [batch_cnt_n]
    int batch_cnt_n = 0;
    pss_raw_cand* raw_pinned = nullptr;       // pinned host staging of downloaded detections
    size_t raw_pinned_n = 0;
    // sifted candidates of the last whole-file search (pss_ctx_take_cands)
    std::vector<pss_cand> last_cands;
    bool has_last = false;
    // multi-file search (pss_search_multi): the group's file bytes, channel-major
    // copies, tables and work lists, and the candidate count of each file of
    // the last group (its lists are in last_cands, file after file)
    DevBuf mf_fil, mf_xcm, mf_work;
    std::vector<int64_t> last_counts;
    std::set<int64_t> mf_seen;   // (transform length, dedispersion variants) the context has run eagerly
    int32_t wait_polls = 0;      // pss_ctx_set_wait_limit: short staging-barrier waits (tests)
    int64_t mf_graphs = 0;       // groups run as a captured graph
    // per-stage event timing (pss_ctx_profile)
    bool prof_on = false;
    struct ProfRec {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
};

// RAII pair of events around one launch when profiling is on.
struct ProfScope {
    Ctx* c;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(Ctx* ctx, int st, cudaStream_t str);
    ~ProfScope();
};

// ---- kernel launchers (each returns cudaGetLastError of its launch) -------
struct PrepArgs {
    const uint8_t* src;   // file bytes on device
    int32_t nchan, nbits, layout;
    int64_t nsamp;
    const int32_t* keep;  // device [Ck] source channel index of each kept row
    int32_t ck;
    uint8_t* xcm;
    int64_t pitch;        // bytes per channel-major row (multiple of 64)
};
cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s);
// Work-list unpack of several files in one launch: item i covers CTAs
// [first, first + CTAs of its grid); items in increasing `first`.
struct PrepItem {
    PrepArgs a;
    int32_t gx;      // tiles along time (the grid's x extent)
    int32_t pad;
    int64_t first;   // first CTA of the item
};
int64_t prep_item_ctas(const PrepArgs& a, int32_t* gx);  // CTAs of one item (sets gx)
cudaError_t launch_prep_multi(const PrepItem* items, int nitems, int64_t total_ctas, cudaStream_t s);

// Let kernel `fn` launch with as much dynamic shared memory as the device
// allows next to its static shared memory (error if `shm` exceeds that).
// Always setting the one maximum, not the launch's own size, keeps
// concurrent host threads that launch the same kernel with different sizes
// from undoing each other's setting.
inline cudaError_t allow_smem(const void* fn, size_t shm) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    const size_t room = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
    if (shm > room) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room);
}

struct DedispArgs {
    const uint8_t* xcm;
    int64_t pitch;
    int32_t ck;
    const int32_t* delays;  // [nb][ck] for this batch
    int32_t nb;             // trials in this batch
    int64_t nv;             // outputs per trial
    int32_t ds;
    float* out_f;           // [nb][out_stride] or null
    int32_t* out_i;         // [nb][out_stride] or null (packed rows use stride nv)
    int64_t out_stride;
    unsigned long long* sums;  // [nb] or null
    int32_t spread;         // max over groups/channels of (dmax - dmin)
    int* err;               // set to 1 if a bounded wait expires (nullable)
    int32_t chunk_kb;       // shared memory for staged channel chunks (0: default)
    int32_t wait_polls;     // > 0: the data waits give up after this many non-blocking polls (tests)
    // two-stage scheme, stage 1: blockIdx.z = subband z sums its own kept
    // channels zsub[z] = (first, count) (ck is then the largest count and
    // sizes the launch), its delays start at delays + first with rows of
    // dstride, and its rows go to out_i + z * zout.  zsub null: one sum over
    // all ck channels, delay rows of ck.
    const int2* zsub;
    int32_t nz;
    int32_t dstride;
    int64_t zout;
};
int dedisp_tile_samples();
int dedisp_group_trials();  // consecutive trials sharing one staged tile
cudaError_t launch_dedisp(const DedispArgs& a, int num_sms, cudaStream_t s);
// Whether launch_dedisp accepts a launch of this delay spread and kept-channel
// count (the host-side checks it makes before launching), so that callers
// can refuse a request before enqueuing any work.
bool dedisp_launch_fits(int32_t spread, int32_t ck, int chunk_kb);
// Work-list dedispersion of several files' trial runs in one launch (exact
// sums into float rows with per-trial sums; one subband): item i covers CTAs
// [first, first + gx * gy); items in increasing `first`.
struct DedispItem {
    DedispArgs a;
    int32_t RW, CC;   // staged row words and channels per chunk (dedisp_item)
    int32_t gx, gy;   // time tiles, groups of trials
    int64_t first;    // first CTA of the item
};
// Fill an item's launch sizes from its arguments (false: the kernel refuses
// them); *shm: the item's dynamic shared memory.
bool dedisp_item(DedispItem* it, int chunk_kb, size_t* shm);
// One launch over items (all with ck <= 256, or all > 256: `wide`); shm the
// largest item's.
cudaError_t launch_dedisp_multi(const DedispItem* items, int nitems, int64_t total_ctas, size_t shm, bool wide,
                                cudaStream_t s);

// Two-stage scheme, stage 2: s_i[t] = sum_b u_{g(i),b}[t + D_b(i)], then the
// ds boxcar, for the nb trials of a batch (k_subband.cu).
struct SubsumArgs {
    const int32_t* u;       // [nsub][group rows][row_stride] stage-1 sums
    int64_t u_zstride;      // elements between subbands
    int64_t u_rowstride;    // elements between group rows
    int64_t u_len;          // valid elements of a row
    int32_t nsub;
    const int32_t* D;       // [nb][nsub] subband delays of the batch's trials
    const int2* grp;        // [group rows] (first trial relative to the tables' start, count)
    int32_t b0rel;          // the batch's first trial relative to the tables' start
    int32_t ngrp;
    int32_t nb;
    int64_t nv;             // outputs per trial
    int32_t ds;
    float* out_f;           // [nb][out_stride] or null
    int32_t* out_i;         // [nb][out_stride] or null
    int64_t out_stride;
    unsigned long long* sums;  // [nb] or null
    int32_t spread;         // max over group rows and subbands of (D max - D min)
    int* err;               // set to 1 if a bounded wait expires (nullable)
    int32_t wait_polls;     // > 0: the data waits give up after this many non-blocking polls (tests)
};
cudaError_t launch_subsum(const SubsumArgs& a, cudaStream_t s);

// Dedispersion of downsampled rows from a per-channel boxcar table
// (k_dedisp_bx.cu): Wt[c][p][m] = sum_{k<ds} x[c][m ds + p + k] (uint16,
// rows of mstride; ds a power of two), then
// s_ds[j] = sum_c Wt[c][d_c mod ds][d_c div ds + j].
constexpr int BX_MAX_DS = 256;  // 255 * ds fits 16 bits
struct BxTableArgs {
    const uint8_t* xcm;
    int64_t pitch;
    int32_t ck;
    int64_t nsamp;
    int32_t lds;       // ds = 2^lds
    int32_t lmt;       // table columns per CTA: 2^lmt = bx_table_cols(ds)
    int64_t mlen;      // columns per phase row: ceil(nsamp / ds)
    int64_t mstride;   // elements between phase rows (>= mlen)
    uint16_t* table;   // [ck][ds][mstride]
};
struct BxArgs {
    const uint16_t* table;
    int64_t mstride;
    int32_t ck;
    int32_t lds;            // ds = 2^lds
    const int32_t* delays;  // [nb][ck]
    int32_t nb;
    int64_t nv;
    float* out_f;           // [nb][out_stride] or null
    int32_t* out_i;         // [nb][out_stride] or null
    int64_t out_stride;
    unsigned long long* sums;  // [nb] or null
};
int bx_table_cols(int ds);
// columns per phase row and the row stride (16-byte rows)
inline int64_t bx_mlen(int64_t nsamp, int ds) { return (nsamp + ds - 1) / ds; }
inline int64_t bx_mstride(int64_t nsamp, int ds) { return (bx_mlen(nsamp, ds) + 7) & ~int64_t(7); }
inline size_t bx_table_bytes(int32_t ck, int64_t nsamp, int ds) {
    return (size_t)ck * (size_t)ds * (size_t)bx_mstride(nsamp, ds) * sizeof(uint16_t);
}
inline bool bx_use(const Tune& t, int ds) {
    return t.bx_min > 0 && ds >= t.bx_min && ds >= 2 && ds <= BX_MAX_DS && (ds & (ds - 1)) == 0;
}
inline int ilog2(int v) {
    int l = 0;
    while ((1 << (l + 1)) <= v) ++l;
    return l;
}
cudaError_t launch_bx_table(const BxTableArgs& a, cudaStream_t s);
cudaError_t launch_dedisp_bx(const BxArgs& a, cudaStream_t s);
// bytes past the last stage-1 row that stage 2's staging copies may read
inline size_t subsum_slack_bytes(int32_t spread) { return (size_t)(1024 + spread + 16) * 4; }

// Single-pulse boxcar search (k_single_pulse.cu).
constexpr int SP_MAXW = 32;         // widths per call
constexpr int SP_MAXWIDTH = 1024;   // largest width
struct SpRaw {
    int32_t dm_idx;
    int32_t w;
    int64_t t;
    int64_t B;
};
struct SpArgs {
    const int32_t* series;  // [nb][stride] exact dedispersed series
    int64_t stride;
    int64_t n;              // samples per trial (N_v)
    int32_t nb;
    int32_t dm0;            // plan index of trial 0
    int32_t w[SP_MAXW];
    int32_t nw, wmax;
    double thr;
    const unsigned long long* s1;  // [nb] sum s
    const unsigned long long* s2;  // [nb] sum s^2
    long long* thr_tab;     // [nb][nw] integer thresholds (written by the moments launch)
    long long max_value;    // largest value a series sample can take (-1: unknown)
    SpRaw* out;
    unsigned long long* count;
    int64_t cap;
};
// moments (into s1, s2, which must be zeroed) then detection
cudaError_t launch_single_pulse(const SpArgs& a, unsigned long long* s1, unsigned long long* s2, cudaStream_t s);
// detection alone (moments already in a.s1, a.s2)
cudaError_t launch_sp_detect_only(const SpArgs& a, cudaStream_t s);
// exact moments alone: s1[b] += sum s, s2[b] += sum s^2 (zero them first)
cudaError_t launch_sp_moments(const int32_t* series, int64_t stride, int64_t n, int32_t nb, unsigned long long* s1,
                              unsigned long long* s2, cudaStream_t s);

// Folding (k_fold.cu): one item per candidate.
struct FoldItem {
    int32_t row;       // series row of the candidate's trial
    int32_t reserved;
    int64_t n;         // samples of that series
    double dt, T;      // sample interval, series span (s)
    double f, fdot;    // candidate frequency (Hz) and drift (Hz/s)
    unsigned long long s1, s2;  // exact moments of the series
};
struct FoldArgs {
    const int32_t* series;  // [rows][stride]
    int64_t stride;
    const FoldItem* items;
    int32_t nbin, nfreq;
    double step_bins;
    long long* prof;        // [items][nfreq][nbin]
    long long* counts;      // [items][nfreq][nbin]
    double* chi2;           // [items][nfreq]
    double* freq;           // [items][nfreq]
};
cudaError_t launch_fold(const FoldArgs& a, int64_t nitems, cudaStream_t s);

struct FftArgs {
    const float* series;              // [nb][series_stride] raw sums (float, exact)
    int64_t series_stride;
    const unsigned long long* sums;   // [nb]
    int64_t nv;
    const int64_t* nv_rows;           // nullable: per-row N_v (rows from several files)
    int64_t nfft;
    int32_t nb;
    float2* bufA;
    float2* bufB;                     // [nb][nfft/2] each
    float2* spec_out;                 // [nb][spec_stride]
    int64_t spec_stride;
    int32_t whiten_block;
    const float2* tw;                 // exp(-2 pi i t / twM), t < twM; twM a multiple of nfft
    int64_t twM;
    int32_t whiten;                   // 0: output the raw half spectrum (DC still zeroed)
    float* gains_out;                 // nullable [nb][gains_stride]: ln 2 / med_b per block
    int64_t gains_stride;
    const float2* ptw[4];             // inter-pass twiddle tables of passes 1.. (fft_pass_plan)
    int32_t fft_variant;              // pass split (fft_pass_plan variant)
    int32_t whiten_form;              // 0: block-per-CTA median, 1: warp-per-block, 2: warp pair per block
    // nullable: whiten and write the zmax 0 plane (2m = 32 taps) here in one pass
    // (whitening blocks of 256, 512 or 1024 bins); the spectrum is then not written
    float* z0_plane;                  // [nb][z0_plane_stride] float2 (|A_k|^2, half-bin power) per bin
    int64_t z0_plane_stride;
    const float* z0_scale1;           // the half-bin taps' normalisation (tap_scale[1])
    float* wscale;                    // [nb][M / whiten_block] scratch: each block's scale
};
cudaError_t launch_twiddles(float2* tw, int64_t n, cudaStream_t s);
// Radices of the passes of an M-point FFT for split `variant` (0 = default);
// returns the pass count (<= 3), or 0 past the last variant.
int fft_pass_plan(int64_t M, int variant, int* rad);
// Instruction-throughput probes (k_probe.cu): per SM clock and per second for
// add3, lop3, prmt, imad, ffma (flops), lop3/imad mix, lds (bytes).
cudaError_t probe_peaks(int sms, cudaStream_t s, uint32_t* sink, unsigned long long* cyc, double per_clk[7],
                        double per_s[7], double* sm_mhz);
cudaError_t launch_pass_twiddles(float2* out, const float2* tw, int64_t twM, int R, int64_t Ns, cudaStream_t s);
cudaError_t launch_fft_whiten(const FftArgs& a, cudaStream_t s, Ctx* prof_ctx);

// Fused spectrum (k_specfused.cu): series -> whitened spectrum -> zmax = 0
// plane for nfft = 2^18, on 16-CTA clusters, one cluster per trial.
struct SpecArgs {
    const float* series;              // [nb][series_stride] raw sums (float, exact)
    int64_t series_stride;
    const unsigned long long* sums;   // [nb]
    int64_t nv;
    int64_t nfft;                     // must be 2^18
    int32_t nb;
    float* plane;                     // [nb][plane_stride] half-bin powers
    int64_t plane_stride;
    const float2* tw;                 // exp(-2 pi i t / twM)
    int64_t twM;
    const float* tap_scale1;          // device: 1/sqrt(E) of the z = 0 odd half-bin taps
};
bool spec_cluster_usable();
cudaError_t launch_spec_cluster(const SpecArgs& a, cudaStream_t s);

struct PlaneArgs {
    const float2* spec;  // [nb][spec_stride] whitened half spectrum (M = nfft/2)
    int64_t spec_stride;
    int64_t nfft;
    int32_t nb;
    float* plane;        // [nb][plane_stride]; row j at j*nfft
    int64_t plane_stride;
    int32_t zmax;
    double dz;
    int32_t extra;
    const float2* taps;  // device template table (zmax > 0)
    const int32_t* tap_off;  // [nz*2] offsets into taps
    const int32_t* tap_m;    // [nz] half-widths
    const float* tap_scale;  // [nz*2] 1/sqrt(E)
    // overlap-save form (zmax > 0): per (row, parity) the spectrum of the
    // taps, [nz][2][fL]; null when the direct form is used
    const float2* ftaps;
    int32_t fL, fV, fM0;     // segment length, valid outputs per segment, lead
    int32_t nz, zrow0;       // rows, and the row with z = 0 exactly (-1: none)
    int32_t form;            // overlap-save FFT: 0 radix 8-8-8-4 (256 threads), 1 radix 16-16-8 (128 threads)
    const float2* tw;        // exp(-2 pi i t / twM)
    int64_t twM;
};
cudaError_t launch_plane(const PlaneArgs& a, cudaStream_t s);

// Overlap-save plane: segment length, and whether it serves (zmax, extra)
// for spectra of M bins (the direct form is used otherwise).
constexpr int PLANE_FFT_L = 2048;
inline bool plane_fft_usable(int32_t zmax, int32_t extra, int64_t M) {
    const int mmax = (zmax + 1) / 2 + extra;
    return zmax > 0 && 4 * mmax <= PLANE_FFT_L && M >= PLANE_FFT_L;
}
struct FftTemplateArgs {
    int32_t nz, zmax, extra;
    double dz;
    const int32_t* tap_m;  // [nz] half-widths
    float2* ftaps;         // out [nz][2][L]
    int32_t L, M0;
};
cudaError_t launch_fft_templates(const FftTemplateArgs& a, cudaStream_t s);

struct TemplateArgs {
    int32_t nz, zmax, extra;
    double dz;
    float2* taps;       // out
    int32_t* tap_off;   // in (host-computed layout, device copy)
    int32_t* tap_m;
    float* tap_scale;   // out
    int32_t total;
};
cudaError_t launch_templates(const TemplateArgs& a, cudaStream_t s);

struct HarmArgs {
    const float* plane;
    int64_t plane_stride;
    int64_t nfft;
    int32_t nz;
    int32_t Z;
    int32_t nb;
    int32_t dm0;        // dm index of batch row 0
    int32_t nstages;    // log2(numharm) + 1
    float thr[6];       // per stage
    int32_t hmin[6];    // per stage
    pss_raw_cand* out;
    unsigned long long* counter;
    int64_t cap;
    int32_t run;        // points per lane of the register-blocked kernel (16 or 8; 0: 16)
    // rows from several files (all nullable): the detection's DM index and file
    // index of each batch row, and each row's per-stage smallest half-bin [nb][8]
    const int32_t* row_dm;
    const int32_t* row_file;
    const int32_t* row_hmin;
};
cudaError_t launch_harm(const HarmArgs& a, cudaStream_t s);


struct RefinePt {
    int32_t trial;    // index into the prepared stage's gains table
    int32_t numharm;
    double dm, r, z;
};
struct RefineArgs {
    const RefinePt* pts;
    const float2* chan_spec;  // [ck][nfft/2] raw per-channel spectra
    const double* dtau;       // [ck] delay per unit DM, seconds
    const float* gains;       // [trials][nblocks] ln 2 / median power
    int64_t nfft;
    int32_t ck;
    int32_t extra;
    int32_t whiten_block;
    int64_t nblocks;
    double T;
    double* power;            // [n]
    double* grad;             // [n][3]: d/dDM, d/dr, d/dz
};
cudaError_t launch_chan_series(const uint8_t* xcm, int64_t pitch, int32_t ck, int64_t nv, int32_t ds, float* out,
                               int64_t out_stride, unsigned long long* sums, cudaStream_t s);
cudaError_t launch_refine_eval(const RefineArgs& a, int64_t n, cudaStream_t s);
int refine_max_taps();

}  // namespace pss

struct pss_ctx : public pss::Ctx {};
struct pss_plan : public pss::Plan {};

namespace pss {
// Raw-detection capacity a pss_batch starts with (it grows on overflow).
constexpr int64_t kBatchInitialCap = (int64_t)1 << 18;
// Argument checks of a whole-file search (pss_batch_create's).
pss_status validate_search(const pss_plan* plan, const pss_fil_desc* fil, const pss_search_cfg* cfg);
// Device bytes a pss_batch for this shape holds with room for dev_cap raw
// detections; host arithmetic only.
size_t search_footprint(const Plan& plan, const pss_fil_desc* fil, const pss_search_cfg* cfg, int64_t dev_cap);
// Device bytes a multi-file search of these files holds (pss_search_multi);
// host arithmetic only.
size_t multi_footprint(const std::vector<const Plan*>& plans, const std::vector<const pss_fil_desc*>& fils,
                       const pss_search_cfg* cfg);
// Device bytes a context holds now.
size_t ctx_device_bytes(const pss_ctx* c);
}  // namespace pss
