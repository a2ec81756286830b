/*
 * pss.h -- C ABI of libpss, a GB300 (sm_103a) library for the per-DM-trial
 * pulsar periodicity search: incoherent dedispersion over a DM plan, a real
 * FFT of every dedispersed series, block-median whitening, an f-fdot
 * (Fourier-domain acceleration) plane, harmonic summing with a sigma
 * threshold, and sifting into a candidate list.
 *
 * The paper ("A PRESTO-based Parallel Pulsar Search Pipeline Used for FAST
 * Drift Scan Data") describes this pipeline as a sequence of programs run
 * once per DM value (Sect. 2, steps 1-7; Sect. 1, the five steps of a pulsar
 * search) with DM plans of the form of Tables 2 and 3.  Each call below
 * names the step it implements.
 *
 * Conventions (all calls):
 *  - Every call returns a pss_status; on failure pss_last_error() returns a
 *    message for the calling thread.  No call aborts the process.
 *  - Pointers documented as "device" must be CUDA device (or managed)
 *    memory of the context's device; "host" pointers are ordinary host
 *    memory (pinned memory makes uploads faster but is not required).
 *  - `stream` is a cudaStream_t passed as void*; NULL means the CUDA
 *    legacy default stream (as for CUDA library calls).  Calls that return
 *    results on the host synchronise that stream before they return; calls
 *    that only write device memory are asynchronous with respect to the
 *    host and ordered on `stream`.
 *  - The caller owns every buffer it passes.  The library owns pss_ctx,
 *    pss_plan and pss_server objects until the matching destroy/free call.
 *  - A pss_ctx may be used by one host thread at a time.
 */
#ifndef PSS_H
#define PSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PSS_OK = 0,
    PSS_EINVAL = -1,     /* invalid argument (message says which)            */
    PSS_ENOMEM = -2,     /* a device or host allocation failed               */
    PSS_ECAP = -3,       /* output capacity too small; *n_out = count needed */
    PSS_ETIMEOUT = -4,   /* a bounded wait expired                           */
    PSS_ECUDA = -5,      /* a CUDA runtime call failed                       */
    PSS_EBUSY = -6,      /* object in use                                    */
    PSS_ENOTREADY = -7   /* result not ready yet                             */
} pss_status;

typedef struct pss_ctx pss_ctx;
typedef struct pss_plan pss_plan;

/* A search-mode filterbank in memory (the paper's test files, Table 1).
 *  nchan, nsamp: channels and time samples.  tsamp_s: sampling time.
 *  fch0_mhz: centre frequency of channel 0; foff_mhz: signed spacing, so
 *  channel c is centred at fch0 + c*foff.
 *  nbits: 8 (one uint8 per sample) or 1 (8 channels per byte, channel c at
 *  bit 7 - c%8 of byte c/8, i.e. most significant bit first; nchan % 8 == 0).
 *  layout: 0 = time-major, file order: sample t of channel c at byte
 *  t*nchan + c (8-bit) or bit as above in row t of nchan/8 bytes (1-bit);
 *  1 = channel-major uint8 [nchan][nsamp] (8-bit only).
 *  chan_mask: optional host array of nchan bytes, nonzero = keep; NULL keeps
 *  every channel (the paper masks RFI with rfifind, Sect. 2 step 1; only a
 *  static mask is supported here). */
typedef struct {
    int32_t nchan;
    int32_t nbits;
    int64_t nsamp;
    double tsamp_s;
    double fch0_mhz;
    double foff_mhz;
    int32_t layout;
    int32_t reserved;
    const uint8_t* chan_mask;
} pss_fil_desc;

/* One row of a dedispersion plan (columns of the paper's Tables 2-3):
 * n_dm trials DM_i = dm_lo + i*dm_step (computed directly in FP64, not by
 * accumulation), the dedispersed series downsampled by ds.  ds must be a
 * power of two between 1 and 1024. */
typedef struct {
    double dm_lo;
    double dm_step;
    int32_t n_dm;
    int32_t ds;
} pss_dd_stage;

/* Search parameters (the paper sets zmax for accelsearch, Sect. 3.2).
 *  zmax: largest |z| (Fourier drift in bins over the series span); 0 = no
 *  acceleration search.  dz: z step; zmax must be a multiple of dz.
 *  numharm: largest harmonic sum (power of two, 1..32).
 *  sigma_thr: single-trial Gaussian-equivalent threshold.
 *  f_lo_hz: lowest fundamental frequency searched.
 *  whiten_block: bins per whitening block (power of two, 64..4096, and a
 *  divisor of nfft/2).  halfwidth_extra: m(z) = ceil(|z|/2) + extra taps
 *  each side (1..64).  min_dm_hits: sifted groups seen in fewer DM trials
 *  are dropped. */
typedef struct {
    int32_t zmax;
    int32_t numharm;
    double dz;
    double sigma_thr;
    double f_lo_hz;
    int32_t whiten_block;
    int32_t halfwidth_extra;
    int32_t min_dm_hits;
    int32_t reserved;
} pss_search_cfg;

/* A raw (unsifted) detection: plane point (h half-bins, row j) at harmonic
 * stage numharm of DM trial dm_idx, with harmonic-summed power `power`. */
typedef struct {
    int32_t dm_idx;
    int32_t numharm;
    int32_t h;
    int32_t j;
    float power;
    int32_t reserved;
} pss_raw_cand;

/* A sifted candidate: fundamental r (bins of the series span T), z (bins),
 * f_hz = r / T, the harmonic stage, summed power, sigma, and the number of
 * DM trials in which the same signal was detected. */
typedef struct {
    int32_t dm_idx;
    int32_t numharm;
    double dm;
    double r;
    double z;
    double f_hz;
    double sigma;
    float power;
    int32_t dm_hits;
    int32_t h;
    int32_t j;
} pss_cand;

/* ---- context ---------------------------------------------------------- */

/* Create a context on CUDA device `device` with a device workspace that
 * grows on demand and is freed by pss_ctx_destroy. */
pss_status pss_ctx_create(int device, pss_ctx** out);
void pss_ctx_destroy(pss_ctx* ctx);
/* Message of the last failed call made by this thread ("" if none). */
const char* pss_last_error(void);
/* Library version string. */
const char* pss_version(void);

/* Failure detection.  Every staging-barrier wait of the dedispersion kernels
 * is bounded: when it runs out the kernel sets an error flag, lets the bulk
 * copies it has in flight land (with the full bound), and leaves without
 * writing; the call then returns PSS_ETIMEOUT and the context stays usable.
 * pss_ctx_set_wait_limit(ctx, polls) with polls > 0 makes those data waits
 * give up after `polls` non-blocking polls on this context (so that a test
 * can make them run out); 0 restores the default bound (2^22 blocking
 * polls).  The limit applies to calls and prepared batches made after it
 * is set.  The paper has no counterpart (its jobs are OS processes). */
pss_status pss_ctx_set_wait_limit(pss_ctx* ctx, int32_t polls);
/* Synchronise `stream` and report (then clear) a bounded-wait failure or a
 * refused launch of the context's kernels since the last report:
 * PSS_ETIMEOUT / PSS_EINVAL, else PSS_OK.  The asynchronous calls
 * (pss_dedisperse) report through this; the calls that synchronise check
 * the flag themselves and discard their results when it is set. */
pss_status pss_ctx_check(pss_ctx* ctx, void* stream);
/* Test hook: the n-th device allocation of the library from now on (any
 * context) fails as if the device were out of memory, and the call that
 * made it returns PSS_ENOMEM; n <= 0 turns the hook off. */
void pss_debug_fail_alloc(int64_t n);

/* Per-stage device-time accounting (tracing).  While enabled, every kernel
 * launch of the search path is bracketed by CUDA events on the stream it is
 * launched on.  Stages: 0 unpack/transpose, 1 dedisperse, 2 FFT passes,
 * 3 R2C + whitening, 4 f-fdot plane, 5 harmonic sum + compaction,
 * 6 boxcar-table builds of the downsampled rows (dedispersion of a row
 * with ds 8-256 is then stage 1).
 * pss_ctx_profile(ctx, 1) enables and resets; (ctx, 0) disables.
 * pss_ctx_profile_read synchronises the recorded events and returns the
 * summed milliseconds and launch counts of each stage (arrays of
 * PSS_NPROF_STAGES), then resets the records.  The paper reports only
 * whole-pipeline wall-clock times (Table 4, Fig. 1); this has no
 * counterpart there. */
#define PSS_NPROF_STAGES 7
pss_status pss_ctx_profile(pss_ctx* ctx, int enable);
pss_status pss_ctx_profile_read(pss_ctx* ctx, double* ms, int64_t* launches);

/* Measured instruction throughputs of a device: the denominators of the
 * integer-arithmetic (dedispersion) and FP32 (template correlation)
 * rooflines.  Each figure comes from one wave of CTAs (4 per SM, 256
 * threads) running 8 independent chains of one instruction kind per thread:
 * add3 = a + b + c (two 32-bit additions), lop3 = (a & b) ^ c, prmt = a
 * byte permute, imad = a * b + c (integer), ffma = FP32 a * b + c (two
 * flops), mix = lop3 and imad alternating (both integer pipes busy: the
 * issue rate), lds = conflict-free 32-bit shared-memory loads (bytes).
 * *_per_clk_sm: per SM clock (cycles counted by clock64); *_per_s: per
 * second over the whole device (CUDA events); sm_mhz: the SM clock the
 * probes ran at.  Allocates a few KiB of device memory and synchronises.
 * The paper has no counterpart (its timings are whole-pipeline CPU wall
 * clock, Table 4). */
typedef struct {
    int32_t sms;
    int32_t reserved;
    double sm_mhz;
    double add3_per_clk_sm, lop3_per_clk_sm, prmt_per_clk_sm, imad_per_clk_sm;
    double ffma_flops_per_clk_sm, mix_per_clk_sm, lds_bytes_per_clk_sm;
    double int32_adds_per_s, lop3_per_s, prmt_per_s, imad_per_s;
    double fp32_flops_per_s, mix_per_s, lds_bytes_per_s;
} pss_peaks;
pss_status pss_measure_peaks(int device, pss_peaks* out);

/* ---- plan (DDplan; Sect. 3.1, Tables 2-3) ------------------------------- */

/* Build the DM grid and the integer delay table of a plan:
 * d[dm][c] = round_half_away(((K*DM) * (1/(f_c*f_c) - 1/(f_ref*f_ref))) / tsamp)
 * evaluated in FP64 in that order, K = 4.148808e3 s MHz^2 pc^-1 cm^3,
 * f_ref = the highest channel frequency.  D = the largest delay; every
 * trial of stage s has N_v = floor((nsamp - D) / ds_s) valid samples and is
 * transformed with nfft = the next power of two >= N_v.
 * Errors: PSS_EINVAL for nsamp <= D, empty stages, bad ds. */
pss_status pss_dd_plan(const pss_fil_desc* fil, const pss_dd_stage* stages, int nstages,
                       pss_plan** out);
/* Stage rows of an automatic dedispersion plan for [dm_lo, dm_hi) (the
 * paper builds its plans with DDplan.py, Sect. 3.1, Tables 2-3; this rule is
 * this library's, from textbook smearing):
 *   t_chan(DM) = 8.3e-6 * DM * |foff| / nu^3,  t_bw(d) = 8.3e-6 * d * BW / nu^3
 * (nu = band centre in GHz, BW = nchan*|foff| MHz, seconds).  A nominal
 * factor v starts at the smallest power of two with v*tsamp >= tres_s
 * (at most ds_max) and doubles per row; a row starting at d0 downsamples by
 * ds = min(v, ds_max), takes the largest step s of 1, 2, 3, 5 x 10^k
 * (0.01 .. 1000) with t_bw(s/2) <= sqrt((ds*tsamp)^2 + t_chan(d0)^2), and
 * holds n = ceil((end - d0)/s - 1e-9) >= 1 trials, end = min(max(DM_sw,
 * d0 + s), dm_hi) with t_chan(DM_sw) = 3.5*v*tsamp; the next row starts at
 * d0 + n*s.  Uses fil's nchan, tsamp_s, fch0_mhz and foff_mhz.
 * out: host array of cap rows; n_out: rows written, or needed with PSS_ECAP.
 * Errors: PSS_EINVAL for a bad descriptor or range, ds_max not a power of
 * two in [1, 1024]. */
pss_status pss_dd_plan_auto(const pss_fil_desc* fil, double dm_lo, double dm_hi, double tres_s, int32_t ds_max,
                            pss_dd_stage* out, int32_t cap, int32_t* n_out);

/* A plan for two-stage (subband) dedispersion, the prepsubband scheme the
 * paper calls faster than one prepdata run per DM (Sect. 5).  Same DM grid
 * as pss_dd_plan; its dedispersion (pss_dedisperse and every search call
 * given this plan) computes, with S = nchan / nsub channels per subband,
 *   stage 1, per group g and subband b:
 *     u_{g,b}[t] = sum over kept channels c of b of x[c][t + e_c(g)],
 *     e_c(g) = round(((K*DM_g) * (1/(f_c*f_c) - 1/(f_b*f_b))) / tsamp),
 *   stage 2, per trial i of group g:
 *     s[t] = sum_b u_{g,b}[t + D_b(i)],
 *     D_b(i) = round(((K*DM_i) * (1/(f_b*f_b) - 1/(f_ref*f_ref))) / tsamp),
 * rounding halves away from zero, then the ds boxcar.  f_b is the highest
 * centre frequency of subband b (channels [b*S, (b+1)*S)); groups are runs
 * of `group` consecutive trials of one stage (the last may be shorter), and
 * DM_g is the DM of a group's middle trial (index first + (n - 1) / 2).
 * The plan's largest delay is D' = max(D, max over trials and channels of
 * e_c(g) + D_b(i)), and N_v follows from D' as in pss_dd_plan.  The sums
 * are exact integers; the scheme approximates each channel's delay (the
 * error is the within-subband delay at DM_i - DM_g plus roundings).
 * Errors: PSS_EINVAL as pss_dd_plan, or nsub not dividing nchan, or group
 * outside [1, 1024].  pss_dedisperse_noalloc refuses such plans. */
pss_status pss_dd_plan_subband(const pss_fil_desc* fil, const pss_dd_stage* stages, int nstages,
                               int32_t nsub, int32_t group, pss_plan** out);
/* The two-stage tables of a plan (nsub == 0 for an exact plan).  Nullable
 * outputs: group_dm [ngroups] doubles; chan_delays [ngroups][nchan] int32
 * (e_c(g), every channel); sub_delays [ndm][nsub] int32 (D_b(i)). */
pss_status pss_plan_subband_info(const pss_plan* plan, int32_t* nsub, int32_t* group, int64_t* ngroups,
                                 double* group_dm, int32_t* chan_delays, int32_t* sub_delays);
/* ndm (total trials) and max_delay (D).  dms (nullable, host, ndm doubles)
 * receives the DM values; delays (nullable, host, ndm*nchan int32,
 * row-major [dm][channel], all channels including masked ones). */
pss_status pss_plan_info(const pss_plan* plan, int64_t* ndm, int64_t* max_delay,
                         double* dms, int32_t* delays);
/* Stage of DM index `dm_idx` and its N_v, nfft, ds. */
pss_status pss_plan_trial_info(const pss_plan* plan, int64_t dm_idx, int32_t* stage,
                               int64_t* nv, int64_t* nfft, int32_t* ds);
void pss_plan_free(pss_plan* plan);

/* ---- dedispersion (Sect. 2 step 2, prepdata/prepsubband) ---------------- */

/* Exact int32 dedispersion of DM trials [dm_begin, dm_end):
 * s[t] = sum over kept channels c of x[c][t + d_c], t < nsamp - D, then
 * s_ds[j] = sum_{k<ds} s[j*ds + k] for j < N_v.
 * data: the file bytes (host if data_on_device == 0, else device).
 * out: device int32; trial i's N_v values start at element
 * sum_{dm_begin <= k < i} N_v(k) (rows packed back to back).
 * Asynchronous: a kernel that gives up (a bounded wait that runs out) is
 * reported by pss_ctx_check or the context's next synchronising call. */
pss_status pss_dedisperse(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil,
                          const void* data, int data_on_device, int64_t dm_begin,
                          int64_t dm_end, int32_t* out, void* stream);

/* Dedispersion for callers that cannot allocate device memory (the paper
 * has no counterpart to this call).  A real-time ingest thread must not call
 * cudaMalloc or cudaFree, which can synchronise the whole device and take
 * unbounded time, and a process whose device memory is already fully reserved
 * by another allocator has none to give; such callers pass their own input
 * and output buffers and this call allocates nothing.
 * Same result and output layout as pss_dedisperse (no context needed), with
 * these differences:
 *  - data_dev must be device memory (there is no upload buffer);
 *  - its scratch (kept-channel list, delays of the requested trials, and a
 *    channel-major copy of the file: about nchan_kept * (nsamp + 1280) bytes
 *    plus 4 * nchan_kept * (dm_end - dm_begin + 1)) lives in one static
 *    device array of PSS_NOALLOC_SCRATCH_BYTES (next to a static 4-byte
 *    error flag); larger requests return PSS_EINVAL with the size needed.
 *    Every GPU that loads the library holds that array until the process
 *    exits;
 *  - the first call on a device looks up the array's device address (set-up
 *    per device, under the current device); make that first call before any
 *    stream capture.  The address is kept for the life of the process: a
 *    caller that resets the device (cudaDeviceReset) invalidates it, and
 *    must not call this entry point on that device afterwards;
 *  - every launch's limits are checked on the host before anything is
 *    enqueued; if a later CUDA step fails, the call waits for `stream` before
 *    it returns the error, so nothing of it is still running;
 *  - every call shares the one array: calls that overlap on the GPU (other
 *    streams, other host threads) race and corrupt each other's results.
 *    Each call overwrites all of the scratch it reads, so nothing carries
 *    over from the previous call;
 *  - it synchronises `stream` before returning. */
#define PSS_NOALLOC_SCRATCH_BYTES (32u << 20)
pss_status pss_dedisperse_noalloc(const pss_plan* plan, const pss_fil_desc* fil, const void* data_dev,
                                  int64_t dm_begin, int64_t dm_end, int32_t* out, void* stream);

/* ---- single-pulse search (Sect. 2 step 7, single_pulse_search.py) ------- */

/* A single-pulse event: boxcar of `width` samples starting at sample t of
 * DM trial dm_idx's dedispersed series (samples of the trial's ds), its
 * exact integer sum and its S/N. */
typedef struct {
    int32_t dm_idx;
    int32_t width;
    int64_t t;
    int64_t boxsum;
    double snr;
} pss_sp_event;

/* Boxcar matched-filter search of the dedispersed series of DM trials
 * [dm_begin, dm_end) (the paper ends its pipeline with a single-pulse
 * search, Sect. 2 step 7; long-period pulsars are found that way, Sect.
 * 5.3).  Per trial, with N = N_v, S1 = sum s, S2 = sum s^2 (exact):
 *   mu = S1/N, sigma = sqrt((S2 - S1*S1/N)/N)                    (FP64, in that order)
 *   B_w[t] = sum_{k<w} s[t+k], 0 <= t <= N - w                   (exact)
 *   detection: B_w[t] >= w*mu + sigma_thr*sigma*sqrt(w), and B_w[t] >
 *   B_w[t'] for t - w < t' < t, B_w[t] >= B_w[t'] for t < t' < t + w;
 *   snr = (B_w[t] - w*mu) / (sigma*sqrt(w));
 * then per trial the detections by snr (descending; ties: smaller width,
 * then earlier) are kept when [t, t + w) overlaps none kept before.  A
 * trial with sigma 0 has no events.  Works with exact and two-stage plans.
 * widths: host array of nwidths (1..32) widths in [1, 1024].
 * out: host array of cap events, sorted by (dm_idx, t).  n_out: the number
 * of events; if it exceeds cap the call returns PSS_ECAP and writes
 * nothing (call again with cap >= n_out).  Synchronises `stream`. */
pss_status pss_single_pulse(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data,
                            int data_on_device, int64_t dm_begin, int64_t dm_end, const int32_t* widths,
                            int32_t nwidths, double sigma_thr, pss_sp_event* out, int64_t cap, int64_t* n_out,
                            void* stream);

/* ---- folding (Sect. 2 step 6, prepfold) -------------------------------- */

/* A candidate to fold: DM trial, frequency (Hz) and drift (Hz/s). */
typedef struct {
    int32_t dm_idx;
    int32_t reserved;
    double f_hz;
    double fdot_hz_s;
} pss_fold_req;

/* Result of folding one candidate: the best trial frequency, its reduced
 * chi-square and its index k in the trial grid. */
typedef struct {
    double f_hz;
    double chi2_red;
    int32_t best;
    int32_t reserved;
} pss_fold_result;

/* Fold each candidate's exact dedispersed series (its DM trial; the paper
 * folds sifted candidates with prepfold, Sect. 2 step 6).  Sample j is at
 * t = j*dt, dt = ds*tsamp; at trial frequency
 *   f_k = f + (k - (nfreq - 1)/2) * (step_bins / T),  k < nfreq,
 * (T = nfft*ds*tsamp of the trial) its phase is phi_j = j*x + j*j*g cycles
 * with x = f_k*dt and g = (0.5*fdot)*(dt*dt) (FP64, in that order), carried
 * in 64-bit fixed point: X = rint(x * 2^64) and G = rint(g * 2^64) modulo
 * 2^64 (rounded half to even from the exact binary values of x and g; a
 * negative g wraps), phase_j = (j*X + j*j*G) mod 2^64, and the bin is
 * floor(phase_j * nbin / 2^64).  This is floor(frac(phi_j) * nbin) except
 * for samples within (j + j*j)*2^-65 cycle of a bin edge (the rounding of X
 * and G); every bin is an exact integer decision.  P_b / n_b: sum / number of the samples of bin b
 * (exact).  With
 * mu = S1/N, var = (S2 - S1*S1/N)/N of the series, chi2_red =
 * sum over bins in order with n_b > 0 of d*d/(n_b*var), d = P_b - n_b*mu,
 * divided by (those bins - 1); 0 when var is 0.  The result is the trial
 * with the largest chi2_red (ties: smaller k).
 * reqs: host [n]; nbin in [2, 1024]; nfreq in [1, 64].
 * profiles, counts: host int64 [n][nbin] (the best trial's); results: host
 * [n].  Works with exact and two-stage plans.  Synchronises `stream`. */
pss_status pss_fold(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data, int data_on_device,
                    const pss_fold_req* reqs, int64_t n, int32_t nbin, int32_t nfreq, double step_bins,
                    int64_t* profiles, int64_t* counts, pss_fold_result* results, void* stream);

/* ---- spectra (Sect. 2 step 3, realfft) ---------------------------------- */

/* Whitened half spectrum of DM trials [dm_begin, dm_end): the dedispersed
 * series minus its mean, zero-padded to nfft, transformed
 * A_k = sum_n y_n exp(-2 pi i k n / nfft) for k < nfft/2, DC set to 0, and
 * every block of whiten_block bins scaled by sqrt(ln 2 / med_b) where med_b
 * is the lower median of |A_k|^2 over the block (DC excluded); a block with
 * median 0 is zeroed.  out: device, interleaved (re, im) float pairs, rows of
 * nfft/2 complex values packed back to back as in pss_dedisperse. */
pss_status pss_spectrum(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil,
                        const void* data, int data_on_device, const pss_search_cfg* cfg,
                        int64_t dm_begin, int64_t dm_end, float* out, void* stream);

/* ---- f-fdot power plane (Sect. 2 step 4 / Sect. 3.2, accelsearch zmax) --- */

/* Normalised power plane P[j][h] = |A(h/2, z_j)|^2 of DM trials
 * [dm_begin, dm_end), z_j = -zmax + j*dz, h in [0, nfft), with
 * A(r, z) = sum_{k=floor(r)-m+1}^{floor(r)+m} A'_k conj(rho(r-k, z)) / sqrt(E),
 * rho(q, z) = integral_0^1 exp(2 pi i ((q - z/2) u + z u^2/2)) du the response
 * of a linearly drifting sinusoid, E the energy of the 2m taps and bins
 * outside [0, nfft/2) taken as 0.  out: device float, per trial n_z*nfft
 * values (row-major [j][h]) packed back to back. */
pss_status pss_power_plane(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil,
                           const void* data, int data_on_device, const pss_search_cfg* cfg,
                           int64_t dm_begin, int64_t dm_end, float* out, void* stream);

/* ---- search (Sect. 2 steps 2-4 fused) ----------------------------------- */

/* Raw detections of DM trials [dm_begin, dm_end): for every harmonic stage
 * n in {1, 2, 4, .., numharm}, S_n(h, j) = sum_{k=1..n} P[j_k][h_k] with
 * h_k = floor((2kh + n) / (2n)), j_k = Z + sgn(j-Z) floor((2k|j-Z| + n)/(2n)),
 * Z = zmax/dz; a point is reported when S_n >= S_thr(n) (the power whose
 * Gamma(n,1) tail probability equals the Gaussian tail at sigma_thr), its
 * fundamental h/(2nT) >= f_lo_hz, and S_n beats all in-plane neighbours of
 * its 3x3 window (exact ties go to the lower linear index j*nfft + h).
 * out: host array of cap entries, sorted by (dm_idx, numharm, j, h).
 * *n_out: the number found; PSS_ECAP (nothing written) if it exceeds cap. */
pss_status pss_search_raw(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil,
                          const void* data, int data_on_device, const pss_search_cfg* cfg,
                          int64_t dm_begin, int64_t dm_end, pss_raw_cand* out, int64_t cap,
                          int64_t* n_out, void* stream);

/* Sifting (Sect. 2 step 5, ACCEL_sift) of raw detections, host only.
 * Each raw point moves to its fundamental r = h/(2n), z = (j-Z) dz / n;
 * within a DM trial, points with |dr| <= 1 and |dz'| <= dz are linked
 * (single linkage) and the highest-sigma member kept (ties: lower n, r, z,
 * DM index); the survivors of all trials are linked the same way, keeping
 * one per group with dm_hits = distinct trials in the group; groups with
 * dm_hits < min_dm_hits are dropped.  Output sorted by (dm_idx, numharm, r, z).
 * PSS_ECAP with *n_out = count needed if cap is too small. */
pss_status pss_sift(const pss_plan* plan, const pss_search_cfg* cfg, const pss_raw_cand* raw,
                    int64_t n_raw, pss_cand* out, int64_t cap, int64_t* n_out);

/* The same sift done the way a pipelined search does it, host only: the raw
 * detections of DM batch b (dm_idx in [dm_bounds[b], dm_bounds[b+1]),
 * b < nbatches; dm_bounds has nbatches + 1 non-decreasing entries) are sifted
 * within their trials batch by batch, the survivors kept ordered by r
 * (zmax 0) or linked to the earlier batches' (zmax > 0), and the across-trial
 * step runs once at the end.  Detections outside every batch are ignored.
 * The result equals pss_sift of the detections inside the batches (single
 * linkage does not depend on the order).  Same output contract as pss_sift. */
pss_status pss_sift_in_batches(const pss_plan* plan, const pss_search_cfg* cfg, const pss_raw_cand* raw,
                               int64_t n_raw, const int64_t* dm_bounds, int32_t nbatches, pss_cand* out,
                               int64_t cap, int64_t* n_out);

/* The whole search of DM trials [dm_begin, dm_end) of one file:
 * pss_search_raw followed by pss_sift.  out: host, cap entries.  The sifted
 * list is also kept in the context (until its next search), so that after
 * PSS_ECAP a caller fetches it with pss_ctx_take_cands instead of searching
 * again. */
pss_status pss_search_dm_batch(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil,
                               const void* data, int data_on_device, const pss_search_cfg* cfg,
                               int64_t dm_begin, int64_t dm_end, pss_cand* out, int64_t cap,
                               int64_t* n_out, void* stream);
/* Copy the sifted candidates of the context's last pss_search_dm_batch
 * (host `out`, cap entries); PSS_ECAP with *n_out = count if cap is too
 * small, PSS_EINVAL if the context has searched nothing. */
pss_status pss_ctx_take_cands(pss_ctx* ctx, pss_cand* out, int64_t cap, int64_t* n_out);

/* ---- candidate refinement (no counterpart in the paper, which folds) ---- */

/* A point of the refinement objective: the trial dm_idx supplies the series
 * span T, nfft and the whitening gains; (dm, r, z) are continuous. */
typedef struct {
    int32_t dm_idx;
    int32_t numharm;
    double dm;
    double r;
    double z;
} pss_refine_point;

/* Prepare refinement for plan stage `stage`: the mean-subtracted spectrum
 * of every kept channel alone (same N_v, ds and nfft as the stage's trials)
 * and the whitening gains ln 2 / med_b of every trial of the stage are kept
 * on the device in the context until the next prepare. */
pss_status pss_refine_prepare(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data,
                              int data_on_device, const pss_search_cfg* cfg, int32_t stage, void* stream);

/* Objective and gradient at n points (host arrays) of the prepared stage:
 *   P_h(DM, r, z) = sum_{k=1..h} g(floor(kr)) |F_k|^2 / E_k,
 *   F_k = sum_c exp(i 2 pi (k r) DM dtau_c / T) sum_q A^c_q conj(rho(kr - q, kz)),
 * q over the 2m(kz) bins nearest kr (as for pss_power_plane), E_k the energy
 * of those taps, dtau_c = K (f_c^-2 - f_ref^-2) the delay per unit DM,
 * g the block's whitening gain in trial dm_idx.  power: n doubles;
 * grad (nullable): 3n doubles (dP/dDM, dP/dr, dP/dz), analytic. */
pss_status pss_refine_eval(pss_ctx* ctx, const pss_plan* plan, const pss_refine_point* pts, int64_t n,
                           double* power, double* grad, void* stream);

/* Gradient ascent (Adam, `iters` steps of size lr in cell units: DM step of
 * the candidate's stage, one bin in r, dz in z; z stays fixed when zmax is
 * 0; at most two cells from the start) on P_h for each candidate (host
 * array).  Each candidate is replaced by the best point visited: dm, r, z,
 * f_hz, power = P_h and its sigma. */
pss_status pss_refine_candidates(pss_ctx* ctx, const pss_plan* plan, const pss_fil_desc* fil, const void* data,
                                 int data_on_device, const pss_search_cfg* cfg, pss_cand* inout, int64_t n,
                                 int32_t iters, double lr, void* stream);

/* Evaluate rho(q_i, z_i) (see pss_power_plane) on the context's GPU in FP64.
 * q, z: host arrays of n doubles; out: host array of 2n doubles (re, im).
 * Exposes the template arithmetic so that it can be checked directly. */
pss_status pss_response(pss_ctx* ctx, const double* q, const double* z, int64_t n, double* out);

/* ---- batched search: one graph launch per file (no paper counterpart) --- */

/* A search prepared for files of one shape (descriptor, plan, cfg): its own
 * context and stream, launch shapes picked by timing (pss_batch_tuning),
 * every device buffer allocated, and the whole kernel sequence of
 * pss_search_dm_batch over all trials of the plan captured into one CUDA
 * graph.  The plan and descriptor are copied; `fil->chan_mask` too.  With a
 * tuned FFT pass split the powers differ from the untuned call's by FP32
 * rounding only. */
typedef struct pss_batch pss_batch;
pss_status pss_batch_create(int device, const pss_plan* plan, const pss_fil_desc* fil, const pss_search_cfg* cfg,
                            pss_batch** out);
/* Search one file of the batch's shape (data: host or device bytes): copy it
 * in, launch the graph, download the detections, sift on the host.  Same
 * result as pss_search_dm_batch over all trials.  gpu_ms (nullable): device
 * time of copy + graph.  Not thread-safe for one batch. */
pss_status pss_batch_run(pss_batch* b, const void* data, int data_on_device, pss_cand* out, int64_t cap,
                         int64_t* n_out, double* gpu_ms);
/* ---- several files in one launch per stage (Sect. 2 parallel versions) -- */

/* One file of a group: its plan (exact, not two-stage), descriptor and bytes
 * (host or device, as the call's data_on_device says). */
typedef struct {
    const pss_plan* plan;
    const pss_fil_desc* fil;
    const void* data;
} pss_multi_file;

/* Search nfiles files of any channel count, sample count, bit depth, layout
 * and DM plan with the same search parameters, as one group: the trials of
 * every file become rows grouped by transform length, and each batch of rows
 * is one launch per stage whose kernels walk a device-side work list (the
 * unpack and dedispersion kernels: items of (file, stage, run of trials,
 * tile); the FFT, whitening, plane and harmonic-sum kernels: rows carrying
 * their file, trial, N_v and f_lo cut).  The sequence runs as one captured
 * CUDA graph (the first group that uses a new transform length on a context
 * runs eagerly, which loads its kernels).  This replaces the paper's
 * process-level parallel versions V2/V3 (Sect. 2) for many files at once.
 * Each file's sifted list is byte-identical to pss_search_dm_batch of that
 * file alone on a context with the same launch shapes.
 * out: host [cap], the lists of file 0, 1, ... back to back; counts: host
 * [nfiles] the length of each; *n_out their total (PSS_ECAP when it exceeds
 * cap: the context keeps the lists for pss_ctx_take_cands, counts are set).
 * PSS_EINVAL for a two-stage plan or arguments pss_search_dm_batch would
 * refuse.  Synchronises `stream`. */
pss_status pss_search_multi(pss_ctx* ctx, const pss_search_cfg* cfg, const pss_multi_file* files, int32_t nfiles,
                            int data_on_device, pss_cand* out, int64_t cap, int64_t* counts, int64_t* n_out,
                            void* stream);
/* Device bytes pss_search_multi holds for this group (host arithmetic, no
 * device): what a server admits a group by. */
pss_status pss_search_multi_footprint(const pss_search_cfg* cfg, const pss_multi_file* files, int32_t nfiles,
                                      size_t* bytes);

/* The sifted candidates of the batch's last pss_batch_run (kept after
 * PSS_ECAP so that they need not be searched again); errors as
 * pss_ctx_take_cands. */
pss_status pss_batch_take_cands(pss_batch* b, pss_cand* out, int64_t cap, int64_t* n_out);
/* Device bytes held by the batch. */
size_t pss_batch_footprint(const pss_batch* b);
/* Launch shapes the batch's autotuner chose (pss_batch_create times each
 * choice on the first <= 256 trials of the shape, timing the stage it
 * changes, and keeps the fastest;
 * the choice is remembered per shape for the life of the process;
 * environment PSS_AUTOTUNE=0 keeps the defaults 0 / 8 / 96 / -1 / 0):
 * fft_split: FFT pass-split variant of the first stage's size (0 = even
 * split; every transform size of a staged plan is tuned on its own, see
 * pss_batch_fft_split), harm_run: points per
 * lane of the harmonic sum (16 or 8), dedisp_kb: shared memory for staged
 * channel chunks (KiB), whiten_form: whitening median per CTA (0), per
 * warp (1), per pair of warps (2) or the default (-1: the pair form for
 * blocks of 256-1024 bins, else per CTA), fused: for zmax 0 and nfft 2^18,
 * FFT + whitening + plane in one
 * thread-block-cluster launch (1) or as separate kernels (0); the fused
 * path is used only where the device can run 16-CTA clusters.  Pointers
 * are nullable. */
pss_status pss_batch_tuning(const pss_batch* b, int32_t* fft_split, int32_t* harm_run, int32_t* dedisp_kb,
                            int32_t* whiten_form, int32_t* fused);
/* The FFT pass split the batch runs for nfft-point series (Sect. 2 step 3,
 * realfft): PSS_EINVAL unless nfft is a power of two >= 128.  Sizes the
 * plan does not use report 0. */
pss_status pss_batch_fft_split(const pss_batch* b, int64_t nfft, int32_t* split);
/* Pass radices of split `split` of the nfft-point real FFT (nfft/2 complex
 * points in the fewest passes of radix 2^5..2^10; split 0 is the even
 * split, larger larger parts first; 1.. the other compositions).  npass:
 * host int32; radices: host int32[4], unused entries 0.  PSS_EINVAL past
 * the last split of the size, and for nfft not a power of two >= 128. */
pss_status pss_fft_split_radices(int64_t nfft, int32_t split, int32_t* npass, int32_t* radices);
/* Pin the FFT pass split a context uses for nfft-point series (what the
 * autotuner of a prepared batch would choose); every later call on the
 * context runs it.  The arithmetic is the same transform, only the FP32
 * rounding order differs.  PSS_EINVAL as pss_fft_split_radices. */
pss_status pss_ctx_set_fft_split(pss_ctx* ctx, int64_t nfft, int32_t split);
/* Device bytes a batch for this shape will hold, computed on the host
 * without a device (what the server admits files by).  PSS_EINVAL for the
 * arguments pss_batch_create would reject. */
pss_status pss_search_footprint(const pss_plan* plan, const pss_fil_desc* fil, const pss_search_cfg* cfg,
                                size_t* bytes);
void pss_batch_free(pss_batch* b);

/* ---- serving: continuous batching of files as they arrive --------------- */

/* A request loop on one device (the paper's drift-scan files arrive one per
 * ~26 s and must each be searched within that budget, Sect. 1).  Up to
 * max_slots files are in flight at once, each on its own stream and batch
 * (kernels of different files overlap on the device); a queued file is
 * admitted, FIFO, when a slot is free and either an idle prepared batch of
 * its shape exists or its device footprint (pss_search_footprint) fits in
 * what is left of hbm_budget_bytes, least recently used idle batches of
 * other shapes being freed to make room (a file larger than the whole
 * budget fails with PSS_ENOMEM).  Thread-safe. */
typedef struct pss_server pss_server;
typedef struct pss_result pss_result;
pss_status pss_server_create(int device, size_t hbm_budget_bytes, int max_slots, pss_server** out);
/* pss_server_create with grouping: with max_group > 1 each slot takes the
 * file at the head of the queue together with the files queued right
 * behind it (same search parameters, exact plans, at most max_group, while
 * the group's footprint fits what is left of the budget) and searches them
 * as one group with pss_search_multi on a context of its own; a two-stage
 * plan runs alone.  Results (per file, by ticket) are the same bytes as the
 * file searched alone with the default launch shapes.  max_group 1 is
 * pss_server_create.  max_group in [1, 1024]. */
pss_status pss_server_create_grouped(int device, size_t hbm_budget_bytes, int max_slots, int max_group,
                                     pss_server** out);
/* Groups a grouped server has run and the files in them. */
pss_status pss_server_group_stats(pss_server* srv, int64_t* groups, int64_t* files);
/* Queue a file (host bytes, copied before return) with its plan stages and
 * search cfg; *ticket identifies the result. */
pss_status pss_submit_file(pss_server* srv, const pss_fil_desc* fil, const void* host_data,
                           const pss_dd_stage* stages, int nstages, const pss_search_cfg* cfg, uint64_t* ticket);
/* pss_submit_file with a two-stage plan (pss_dd_plan_subband(fil, stages,
 * nstages, nsub, group)); files of the same shape and plan share prepared
 * batches as with pss_submit_file.  PSS_EINVAL for nsub <= 0 and for what
 * pss_dd_plan_subband rejects. */
pss_status pss_submit_file_subband(pss_server* srv, const pss_fil_desc* fil, const void* host_data,
                                   const pss_dd_stage* stages, int nstages, int32_t nsub, int32_t group,
                                   const pss_search_cfg* cfg, uint64_t* ticket);
/* Wait up to timeout_ms for a ticket's result: PSS_ENOTREADY if timeout_ms
 * is 0 and it is not ready, PSS_ETIMEOUT if the wait expires.  The result is
 * handed over once (free it with pss_result_free). */
pss_status pss_poll(pss_server* srv, uint64_t ticket, int timeout_ms, pss_result** out);
/* The file's outcome (PSS_OK or the error it met), its sifted candidates
 * (valid until pss_result_free), and submit-to-ready latency in seconds. */
pss_status pss_result_cands(const pss_result* r, const pss_cand** c, int64_t* n, double* latency_s);
void pss_result_free(pss_result* r);
/* Completed files, and the 50th / 99th percentile latency over them (s). */
pss_status pss_server_stats(pss_server* srv, int64_t* completed, double* p50_s, double* p99_s, size_t* bytes_in_use);
void pss_server_destroy(pss_server* srv);

/* Significance of a harmonic sum: -Phi^-1(Q(n, S)) with
 * Q(n, S) = exp(-S) sum_{j<n} S^j / j!, and its inverse (the threshold). */
double pss_sigma_of_power(int32_t numharm, double power);
double pss_power_threshold(int32_t numharm, double sigma);

#ifdef __cplusplus
}
#endif
#endif /* PSS_H */
