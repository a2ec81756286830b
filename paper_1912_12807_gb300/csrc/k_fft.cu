// Batched real FFT of the dedispersed series and block-median whitening
// (paper Sect. 2 step 3, realfft; whitening is not described in the paper).
//
// A real series y of length nfft is packed as z[n] = y[2n] + i y[2n+1] and
// transformed with an M = nfft/2 point complex FFT; the half spectrum
//   A_k = (Z_k + conj Z_{M-k}) / 2 - (i/2) e^{-2 pi i k / nfft} (Z_k - conj Z_{M-k})
// is formed in the whitening kernel.
//
// The complex FFT is a Stockham auto-sort FFT with a few large-radix passes
// (radix R = 32..1024, product = M).  In the pass with running length Ns,
// element j + r*M/R (r < R) of each of the M/R columns is multiplied by
// exp(-2 pi i r (j mod Ns) / (Ns R)), transformed by an R-point DFT and
// written to (j / Ns) * Ns * R + (j mod Ns) + r * Ns.  A CTA owns TJ = 8
// consecutive columns, reads them as contiguous 64-byte rows, does the
// R-point DFT in shared memory with radix-8 Stockham sub-stages (one radix-2
// or radix-4 sub-stage first when log2 R is not a multiple of 3), in place
// (inputs of a sub-stage are held in registers across a barrier), and writes
// contiguous rows.  Two passes cover M <= 2^20, three up to 2^24.  All twiddle factors
// come from one table exp(-2 pi i t / Mt) (t < Mt, computed in FP64 and
// rounded to FP32), read with stride Mt / P for a P-th root of unity.
//
// The first pass also subtracts the series mean (exact integer sum / N_v,
// split into an integer and a fractional part so the FP32 subtraction is
// exact up to one rounding) and zero-pads past N_v.
#include <math.h>
#include <stdlib.h>

#include "bulk.cuh"
#include "fft_small.cuh"
#include "whiten.cuh"
#include "pss_internal.h"

namespace pss {

namespace {

constexpr int TJ = 8;        // columns per CTA
constexpr int TJP = TJ + 1;  // padded shared-memory row (bank spread)
constexpr int NT = 256;      // threads per CTA

// One Stockham sub-stage of radix RR on the R-point DFTs of TJ columns,
// in place in shared memory ([r * TJP + jj]), running span ns: every thread
// reads its butterflies' inputs into registers, the block synchronises, and
// the results are written back.  The twiddle exp(-2 pi i q k / (RR ns)) is
// twt[q ns + k] (a table per sub-stage, q-major so that the lanes of a warp,
// which hold consecutive k, read consecutive words).
template <int R, int RR>
__device__ __forceinline__ void substage(float2* buf, const float2* twt, int ns) {
    constexpr int NB = R / RR * TJ;
    constexpr int PER = (NB + NT - 1) / NT;
    float2 x[PER][RR];
    int dst[PER];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int e = threadIdx.x + p * NT;
        if (NB % NT == 0 || e < NB) {
            const int jj = e % TJ, b = e / TJ;
            const int k = b & (ns - 1);
#pragma unroll
            for (int q = 0; q < RR; ++q) {
                x[p][q] = buf[(b + q * (R / RR)) * TJP + jj];
                if (q && k) x[p][q] = cmul(x[p][q], twt[q * ns + k]);
            }
            dst[p] = ((b - k) * RR + k) * TJP + jj;
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int e = threadIdx.x + p * NT;
        if (NB % NT == 0 || e < NB) {
            dft_small<RR>(x[p]);
#pragma unroll
            for (int q = 0; q < RR; ++q) buf[dst[p] + q * ns * TJP] = x[p][q];
        }
    }
    __syncthreads();
}

// Sub-stage plan of an R-point DFT: one radix-2 or radix-4 sub-stage first
// when log2 R is not a multiple of 3, then radix 8.  Sub-stages after the
// first have running span ns > 1 and a twiddle table of RR * ns entries.
template <int R>
struct SubPlan {
    static constexpr int LOG = (R == 32) ? 5 : (R == 64) ? 6 : (R == 128) ? 7 : (R == 256) ? 8 : (R == 512) ? 9 : 10;
    static constexpr int FIRST = (LOG % 3 == 1) ? 2 : (LOG % 3 == 2) ? 4 : 8;
    // total twiddle-table entries: sum of 8 ns over the radix-8 sub-stages with ns > 1
    static constexpr int table_size() {
        int t = 0;
        for (int ns = FIRST; ns < R; ns *= 8) t += 8 * ns;
        return t;
    }
};

// Fill the sub-stage twiddle tables from the global table exp(-2 pi i t / twM).
template <int R>
__device__ void load_subtables(float2* twt, const float2* tw, int64_t twM) {
    const int64_t tstride = twM / R;
    int off = 0;
    for (int ns = SubPlan<R>::FIRST; ns < R; ns *= 8) {
        for (int i = threadIdx.x; i < 8 * ns; i += NT) {
            const int q = i / ns, k = i - q * ns;
            twt[off + i] = tw[(int64_t)(q * k * (R / (8 * ns))) * tstride];
        }
        off += 8 * ns;
    }
}

// R-point DFTs of TJ columns held in buf (in place).
template <int R>
__device__ void smem_dft(float2* buf, const float2* twt) {
    constexpr int FIRST = SubPlan<R>::FIRST;
    if constexpr (FIRST == 2) substage<R, 2>(buf, twt, 1);
    else if constexpr (FIRST == 4) substage<R, 4>(buf, twt, 1);
    else substage<R, 8>(buf, twt, 1);
    int off = 0;
    for (int ns = FIRST; ns < R; ns *= 8) {
        substage<R, 8>(buf, twt + off, ns);
        off += 8 * ns;
    }
}

struct PassArgs {
    const float2* in;          // [nb][in_stride] complex (null on the first pass)
    int64_t in_stride;
    const float* series;       // first pass: real series [nb][series_stride]
    int64_t series_stride;
    const unsigned long long* sums;
    int64_t nv;
    const int64_t* nv_rows;    // first pass: per-row N_v (nullable: every row has nv)
    float2* out;
    int64_t out_stride;
    int64_t M;
    int64_t Ns;
    const float2* tw;          // exp(-2 pi i t / twM)
    int64_t twM;
    const float2* ptw;         // later passes: [R][Ns] inter-pass twiddles tw[r k twM / (Ns R)]
};

// N_v of batch row b (per-row lengths when the rows come from several files)
__device__ __forceinline__ int64_t row_nv(const PassArgs& a, int b) { return a.nv_rows ? a.nv_rows[b] : a.nv; }

template <int R>
__global__ void __launch_bounds__(NT) k_fft_pass(const __grid_constant__ PassArgs a) {
    extern __shared__ float2 sm[];
    float2* bufA = sm;
    float2* twt = sm + R * TJP;  // sub-stage twiddle tables
    const int b = blockIdx.y;
    const int64_t ncol = a.M / R;
    const int64_t j0 = (int64_t)blockIdx.x * TJ;
    const bool first = (a.series != nullptr);
    load_subtables<R>(twt, a.tw, a.twM);

    if (first) {
        // mean = sum / N_v in FP64 (once per CTA: FP64 is slow), split as integer + fraction
        __shared__ float s_mu[2];
        if (threadIdx.x == 0) {
            const double mu = (double)a.sums[b] / (double)row_nv(a, b);
            const double mi = rint(mu);
            s_mu[0] = (float)mi;
            s_mu[1] = (float)(mu - mi);
        }
        __syncthreads();
        const float mu_i = s_mu[0], mu_f = s_mu[1];
        const float* s = a.series + (int64_t)b * a.series_stride;
        const int64_t nv = row_nv(a, b);
#pragma unroll
        for (int e = threadIdx.x; e < R * TJ; e += NT) {
            const int jj = e % TJ, r = e / TJ;
            const int64_t j = j0 + jj;
            float2 x = make_float2(0.f, 0.f);
            if (j < ncol) {
                const int64_t n = j + (int64_t)r * ncol;
                if (2 * n + 1 < nv) {
                    const float2 v = *reinterpret_cast<const float2*>(s + 2 * n);
                    x = make_float2((v.x - mu_i) - mu_f, (v.y - mu_i) - mu_f);
                } else if (2 * n < nv) {
                    x.x = (s[2 * n] - mu_i) - mu_f;
                }
            }
            bufA[r * TJP + jj] = x;
        }
    } else {
        const float2* in = a.in + (int64_t)b * a.in_stride;
#pragma unroll
        for (int e = threadIdx.x; e < R * TJ; e += NT) {
            const int jj = e % TJ, r = e / TJ;
            const int64_t j = j0 + jj;
            float2 x = make_float2(0.f, 0.f);
            if (j < ncol) {
                x = in[j + (int64_t)r * ncol];
                const int64_t k = j & (a.Ns - 1);  // Ns: a power of two
                // table laid out like the data: consecutive columns read consecutive words
                if (k && r) x = cmul(x, a.ptw[(int64_t)r * a.Ns + k]);
            }
            bufA[r * TJP + jj] = x;
        }
    }
    __syncthreads();
    smem_dft<R>(bufA, twt);
    const float2* res = bufA;
    float2* o = a.out + (int64_t)b * a.out_stride;
    if (a.Ns == 1) {
        for (int e = threadIdx.x; e < R * TJ; e += NT) {
            const int r = e % R, jj = e / R;
            const int64_t j = j0 + jj;
            if (j < ncol) o[j * R + r] = res[r * TJP + jj];
        }
    } else {
        for (int e = threadIdx.x; e < R * TJ; e += NT) {
            const int jj = e % TJ, r = e / TJ;
            const int64_t j = j0 + jj;
            if (j < ncol) {
                const int64_t k = j & (a.Ns - 1);  // Ns: a power of two
                o[(j / a.Ns) * a.Ns * R + k + (int64_t)r * a.Ns] = res[r * TJP + jj];
            }
        }
    }
}

// ---- double-buffered form -------------------------------------------------
// The same pass, but a CTA walks `tpc` consecutive tiles of one trial and
// brings tile t+1 into a second shared-memory buffer with asynchronous
// 8-byte copies (cp.async, zero-filled past the data) while it transforms
// and writes tile t, so global-load latency overlaps the sub-stages.  The
// mean subtraction and padding of the first pass, and the inter-pass
// twiddles of later passes (prefetched into registers one tile ahead), are
// applied in shared memory once a tile has landed.  Same arithmetic in the
// same order as k_fft_pass: the results are bit-identical.

template <int R>
__device__ __forceinline__ void issue_tile(const PassArgs& a, int b, int64_t j0, float2* buf) {
    const int64_t ncol = a.M / R;
    if (a.series != nullptr) {
        const int64_t nv = row_nv(a, b);
        const float* s = a.series + (int64_t)b * a.series_stride;
#pragma unroll
        for (int i = 0; i < R * TJ / NT; ++i) {
            const int e = threadIdx.x + i * NT;
            const int jj = e % TJ, r = e / TJ;
            const int64_t j = j0 + jj;
            const int64_t n = j + (int64_t)r * ncol;
            // both samples, the first only (the odd tail), or none (zeros)
            const uint32_t nbytes = (j < ncol && 2 * n + 1 < nv) ? 8u : ((j < ncol && 2 * n < nv) ? 4u : 0u);
            cp_async8(buf + r * TJP + jj, nbytes ? (const void*)(s + 2 * n) : (const void*)s, nbytes);
        }
    } else {
        const float2* in = a.in + (int64_t)b * a.in_stride;
#pragma unroll
        for (int i = 0; i < R * TJ / NT; ++i) {
            const int e = threadIdx.x + i * NT;
            const int jj = e % TJ, r = e / TJ;
            const int64_t j = j0 + jj;
            const bool ok = j < ncol;
            cp_async8(buf + r * TJP + jj, ok ? (const void*)(in + j + (int64_t)r * ncol) : (const void*)in,
                      ok ? 8u : 0u);
        }
    }
}

template <int R>
__device__ __forceinline__ void load_ptw(const PassArgs& a, int64_t j0, float2 (&w)[R * TJ / NT]) {
    const int64_t ncol = a.M / R;
#pragma unroll
    for (int i = 0; i < R * TJ / NT; ++i) {
        const int e = threadIdx.x + i * NT;
        const int jj = e % TJ, r = e / TJ;
        const int64_t j = j0 + jj;
        const int64_t k = j & (a.Ns - 1);  // Ns: a power of two
        w[i] = (j < ncol && k && r) ? a.ptw[(int64_t)r * a.Ns + k] : make_float2(1.f, 0.f);
    }
}

// CTAs per SM the register budget is sized for: shared memory allows about
// four of the radix <= 256 forms and two of the 512 form
template <int R>
constexpr int db_min_blocks() { return R <= 256 ? 4 : (R == 512 ? 2 : 1); }

template <int R, bool FIRST>
__global__ void __launch_bounds__(NT, db_min_blocks<R>()) k_fft_pass_db(const __grid_constant__ PassArgs a, int tpc) {
    extern __shared__ float2 sm[];
    float2* twt = sm + 2 * R * TJP;  // sub-stage twiddle tables
    const int b = blockIdx.y;
    const int64_t ncol = a.M / R;
    const int64_t ntile = (ncol + TJ - 1) / TJ;
    const int64_t tile0 = (int64_t)blockIdx.x * tpc;
    const int64_t tile1 = min(ntile, tile0 + tpc);
    constexpr bool first = FIRST;
    issue_tile<R>(a, b, tile0 * TJ, sm);
    cp_async_commit();
    load_subtables<R>(twt, a.tw, a.twM);
    float mu_i = 0.f, mu_f = 0.f;
    const int64_t nv_b = first ? row_nv(a, b) : 0;
    if (first) {
        // mean = sum / N_v in FP64 (once per CTA: FP64 is slow), split as integer + fraction
        __shared__ float s_mu[2];
        if (threadIdx.x == 0) {
            const double mu = (double)a.sums[b] / (double)row_nv(a, b);
            const double mi = rint(mu);
            s_mu[0] = (float)mi;
            s_mu[1] = (float)(mu - mi);
        }
        __syncthreads();
        mu_i = s_mu[0];
        mu_f = s_mu[1];
    }
    float2 w[FIRST ? 1 : R * TJ / NT];
    if constexpr (!FIRST) load_ptw<R>(a, tile0 * TJ, w);
    float2* o = a.out + (int64_t)b * a.out_stride;
    for (int64_t t = tile0; t < tile1; ++t) {
        float2* cur = sm + ((t - tile0) & 1) * (R * TJP);
        const int64_t j0 = t * TJ;
        if (t + 1 < tile1) {
            issue_tile<R>(a, b, j0 + TJ, sm + ((t + 1 - tile0) & 1) * (R * TJP));
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        // fix-up in place: mean and padding (first pass) or inter-pass twiddles
#pragma unroll
        for (int i = 0; i < R * TJ / NT; ++i) {
            const int e = threadIdx.x + i * NT;
            const int jj = e % TJ, r = e / TJ;
            float2& x = cur[r * TJP + jj];
            if constexpr (FIRST) {
                const int64_t j = j0 + jj;
                const int64_t n = j + (int64_t)r * ncol;
                float2 v = make_float2(0.f, 0.f);
                if (j < ncol) {
                    if (2 * n + 1 < nv_b) v = make_float2((x.x - mu_i) - mu_f, (x.y - mu_i) - mu_f);
                    else if (2 * n < nv_b) v.x = (x.x - mu_i) - mu_f;
                }
                x = v;
            } else {
                const int64_t j = j0 + jj;
                if (j < ncol && (j & (a.Ns - 1)) && r) x = cmul(x, w[i]);
            }
        }
        if constexpr (!FIRST) {
            if (t + 1 < tile1) load_ptw<R>(a, j0 + TJ, w);
        }
        __syncthreads();
        smem_dft<R>(cur, twt);
        const float2* res = cur;
        if (a.Ns == 1) {
            for (int e = threadIdx.x; e < R * TJ; e += NT) {
                const int r = e % R, jj = e / R;
                const int64_t j = j0 + jj;
                if (j < ncol) o[j * R + r] = res[r * TJP + jj];
            }
        } else {
            for (int e = threadIdx.x; e < R * TJ; e += NT) {
                const int jj = e % TJ, r = e / TJ;
                const int64_t j = j0 + jj;
                if (j < ncol) {
                    const int64_t k = j & (a.Ns - 1);  // Ns: a power of two
                    o[(j / a.Ns) * a.Ns * R + k + (int64_t)r * a.Ns] = res[r * TJP + jj];
                }
            }
        }
        __syncthreads();
    }
}

// Tiles per CTA of the double-buffered passes (PSS_FFT_TPC overrides) and
// whether they are used (PSS_FFT_DB=0 keeps the single-buffered form).
int fft_tpc() {
    static const int v = [] {
        const char* e = getenv("PSS_FFT_TPC");
        const int x = e ? atoi(e) : 4;
        return x < 1 ? 1 : x;
    }();
    return v;
}
// PSS_FFT_DB=0 / 1 forces the single- / double-buffered passes; by default
// the double-buffered form runs for spectra of up to 2^17 bins, where it is
// measured faster (a 2^18-point real series: 1.94 -> 1.73 ms per 1001
// trials), and the single-buffered one above (2^22 bins: 58.0 against 59.5 ms).
bool fft_db(int64_t M) {
    static const int v = [] {
        const char* e = getenv("PSS_FFT_DB");
        return e ? (e[0] == '1' ? 1 : 0) : -1;
    }();
    return v < 0 ? M <= (int64_t(1) << 17) : v == 1;
}

template <int R>
cudaError_t run_pass(const PassArgs& p, int nb, cudaStream_t s) {
    if (fft_db(p.M)) {
        const size_t shm2 = (size_t)(2 * R * TJP + SubPlan<R>::table_size()) * sizeof(float2);
        const void* k = p.series ? (const void*)k_fft_pass_db<R, true> : (const void*)k_fft_pass_db<R, false>;
        cudaError_t e = allow_smem(k, shm2);
        if (e != cudaSuccess) return e;
        const int64_t ntile = (p.M / R + TJ - 1) / TJ;
        const int tpc = (int)std::max<int64_t>(1, std::min<int64_t>(fft_tpc(), ntile));
        dim3 grid((unsigned)((ntile + tpc - 1) / tpc), (unsigned)nb);
        if (p.series) k_fft_pass_db<R, true><<<grid, NT, shm2, s>>>(p, tpc);
        else k_fft_pass_db<R, false><<<grid, NT, shm2, s>>>(p, tpc);
        return cudaGetLastError();
    }
    const size_t shm = (size_t)(R * TJP + SubPlan<R>::table_size()) * sizeof(float2);
    cudaError_t e = allow_smem((const void*)k_fft_pass<R>, shm);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((p.M / R + TJ - 1) / TJ), (unsigned)nb);
    k_fft_pass<R><<<grid, NT, shm, s>>>(p);
    return cudaGetLastError();
}

// ---- register-radix form ----------------------------------------------------
// The same pass with its R-point DFTs split into two or three register
// sub-stages (radix 4, 8 or 16) whose first reads the columns straight from
// global memory (mean, padding or inter-pass twiddles applied in registers)
// and whose last writes the results straight to global memory, so an
// element crosses shared memory once (two sub-stages) or twice (three)
// instead of being staged, fixed up, transformed in place and read back.
// Sub-stage with radix RR and running span ns (Stockham, as in `substage`):
// butterfly b takes elements b + q R/RR (q < RR) of its column, twiddled by
// exp(-2 pi i q (b mod ns) / (RR ns)), and writes the RR-point DFT to
// ((b - b mod ns) RR + b mod ns) + q ns; in the last sub-stage ns RR = R and
// the result of butterfly b, output q, is frequency b + q R/RR.
// A CTA owns RT columns; its threads take butterflies column-fastest
// (coalesced column reads, and writes of later passes), except the last
// sub-stage of the first pass (Ns = 1), whose outputs are contiguous in
// frequency: there the threads take butterflies b-fastest.
template <int R>
struct RrPlan {
    // sub-stage radices: first, middle (0: none), last
    static constexpr int A = (R == 32) ? 4 : (R == 64) ? 8 : (R == 128) ? 16 : (R == 256) ? 16 : (R == 512) ? 8 : 16;
    static constexpr int B = (R == 512 || R == 1024) ? 8 : 0;
    static constexpr int C = R / A / (B ? B : 1);
    static constexpr int RT = (R == 32) ? 32 : (R == 64 || R == 128) ? 16 : 8;  // columns per CTA
    static constexpr int NTR = (R >= 512) ? 256 : 128;                       // threads
    // CTAs per SM the register budget must allow: the counts the compiler reaches by itself,
    // except radix 128 (the passes of 2^20-2^22-point transforms), held to 48 registers
    static constexpr int MINB = (R == 32) ? 16 : (R == 64) ? 12 : (R == 128) ? 10 : (R == 256) ? 9 : (R == 512) ? 4 : 2;
    static constexpr int RTP = RT + 1;
    // twiddle entries of the sub-stages after the first: B * A (middle) + C * (R / C)
    static constexpr int TW = (B ? B * A : 0) + R;
};

template <int R, int RR, int RT, int NTR>
__device__ __forceinline__ void rr_mid(float2* buf, const float2* twt, int ns) {
    constexpr int NB = R / RR * RT;
    constexpr int PER = (NB + NTR - 1) / NTR;
    float2 x[PER][RR];
    int dst[PER];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int e = threadIdx.x + p * NTR;
        if (NB % NTR == 0 || e < NB) {
            const int jj = e % RT, b = e / RT;
            const int k = b & (ns - 1);
#pragma unroll
            for (int q = 0; q < RR; ++q) {
                x[p][q] = buf[(b + q * (R / RR)) * (RT + 1) + jj];
                if (q && k) x[p][q] = cmul(x[p][q], twt[q * ns + k]);
            }
            dst[p] = ((b - k) * RR + k) * (RT + 1) + jj;
        }
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int e = threadIdx.x + p * NTR;
        if (NB % NTR == 0 || e < NB) {
            dft_any<RR>(x[p]);
#pragma unroll
            for (int q = 0; q < RR; ++q) buf[dst[p] + q * ns * (RT + 1)] = x[p][q];
        }
    }
    __syncthreads();
}

template <int R, bool FIRST>
__global__ void __launch_bounds__(RrPlan<R>::NTR, RrPlan<R>::MINB) k_fft_pass_rr(const __grid_constant__ PassArgs a) {
    using P = RrPlan<R>;
    constexpr int A = P::A, B = P::B, C = P::C, RT = P::RT, RTP = P::RTP, NTR = P::NTR;
    extern __shared__ float2 sm[];
    float2* buf = sm;               // [R][RTP]
    float2* twt = sm + R * RTP;     // middle table [B * A] (q-major), then the last [C * (R / C)]
    const int b = blockIdx.y;
    const int64_t ncol = a.M / R;
    const int64_t j0 = (int64_t)blockIdx.x * RT;
    // sub-stage twiddle tables from the global table exp(-2 pi i t / twM)
    {
        const int64_t tstride = a.twM / R;
        int off = 0;
        if constexpr (B != 0) {
            // middle: ns = A, radix B: exp(-2 pi i q k / (B A)), q < B, k < A
            for (int i = threadIdx.x; i < B * A; i += NTR) {
                const int q = i / A, k = i - q * A;
                twt[i] = a.tw[(int64_t)(q * k * (R / (B * A))) * tstride];
            }
            off = B * A;
        }
        // last: ns = R / C, radix C: exp(-2 pi i q k / R), q < C, k < R / C
        for (int i = threadIdx.x; i < R; i += NTR) {
            const int q = i / (R / C), k = i - q * (R / C);
            twt[off + i] = a.tw[(int64_t)(q * k) * tstride];
        }
    }
    // first sub-stage: radix A from global memory, ns = 1 (no twiddles inside the DFT)
    {
        float mu_i = 0.f, mu_f = 0.f;
        int64_t nv = 0;
        if constexpr (FIRST) {
            __shared__ float s_mu[2];
            if (threadIdx.x == 0) {
                // mean = sum / N_v in FP64 (once per CTA), split as integer + fraction
                const double mu = (double)a.sums[b] / (double)row_nv(a, b);
                const double mi = rint(mu);
                s_mu[0] = (float)mi;
                s_mu[1] = (float)(mu - mi);
            }
            __syncthreads();
            mu_i = s_mu[0];
            mu_f = s_mu[1];
            nv = row_nv(a, b);
        }
        constexpr int NB = R / A * RT;
        constexpr int PER = (NB + NTR - 1) / NTR;
        const float* sr = FIRST ? a.series + (int64_t)b * a.series_stride : nullptr;
        const float2* in = FIRST ? nullptr : a.in + (int64_t)b * a.in_stride;
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int e = threadIdx.x + p * NTR;
            if (NB % NTR == 0 || e < NB) {
                const int jj = e % RT, bb = e / RT;
                const int64_t j = j0 + jj;
                float2 x[A];
#pragma unroll
                for (int q = 0; q < A; ++q) {
                    const int r = bb + q * (R / A);
                    float2 v = make_float2(0.f, 0.f);
                    if (j < ncol) {
                        const int64_t n = j + (int64_t)r * ncol;
                        if constexpr (FIRST) {
                            if (2 * n + 1 < nv) {
                                const float2 w = *reinterpret_cast<const float2*>(sr + 2 * n);
                                v = make_float2((w.x - mu_i) - mu_f, (w.y - mu_i) - mu_f);
                            } else if (2 * n < nv) {
                                v.x = (sr[2 * n] - mu_i) - mu_f;
                            }
                        } else {
                            v = in[n];
                            const int64_t k = j & (a.Ns - 1);  // Ns: a power of two
                            if (k && r) v = cmul(v, a.ptw[(int64_t)r * a.Ns + k]);
                        }
                    }
                    x[q] = v;
                }
                dft_any<A>(x);
#pragma unroll
                for (int q = 0; q < A; ++q) buf[(bb * A + q) * RTP + jj] = x[q];
            }
        }
        __syncthreads();
    }
    if constexpr (B != 0) rr_mid<R, B, RT, NTR>(buf, twt, A);
    // last sub-stage: radix C, ns = R / C, straight to global memory
    {
        constexpr int NS = R / C;
        const float2* tl = twt + (B ? B * A : 0);
        constexpr int NB = R / C * RT;
        constexpr int PER = (NB + NTR - 1) / NTR;
        float2* o = a.out + (int64_t)b * a.out_stride;
        const bool ns1 = a.Ns == 1;
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int e = threadIdx.x + p * NTR;
            if (NB % NTR == 0 || e < NB) {
                // Ns = 1: butterflies b-fastest (contiguous frequencies); else column-fastest
                const int jj = ns1 ? e / NS : e % RT;
                const int bb = ns1 ? e % NS : e / RT;
                float2 x[C];
#pragma unroll
                for (int q = 0; q < C; ++q) {
                    x[q] = buf[(bb + q * NS) * RTP + jj];
                    if (q && bb) x[q] = cmul(x[q], tl[q * NS + bb]);
                }
                dft_any<C>(x);
                const int64_t j = j0 + jj;
                if (j < ncol) {
                    if (ns1) {
#pragma unroll
                        for (int q = 0; q < C; ++q) o[j * R + bb + q * NS] = x[q];
                    } else {
                        const int64_t kc = j & (a.Ns - 1);
                        float2* oo = o + (j / a.Ns) * a.Ns * R + kc;
#pragma unroll
                        for (int q = 0; q < C; ++q) oo[(int64_t)(bb + q * NS) * a.Ns] = x[q];
                    }
                }
            }
        }
    }
}

// ---- register-radix form with staged, double-buffered tiles -----------------
// The same pass as k_fft_pass_rr, but a CTA walks `tpc` consecutive column
// tiles of one trial: while it transforms tile t, tile t+1 (and, after the
// first pass, the tile's inter-pass twiddles, which have the same shape:
// rows r, columns (j mod Ns) .. + RT) comes into shared memory by
// asynchronous 8-byte copies (zero-filled past the data).  The first
// sub-stage reads the landed tile, mean, padding or twiddles applied in
// registers as k_fft_pass_rr does; the tile's buffer then holds the later
// sub-stages, and the sub-stage twiddle tables are built once per CTA.
// Same operations in the same order: bit-identical to k_fft_pass_rr.
template <int R, bool FIRST>
struct RrdbPlan {
    static constexpr int TS = R * RrPlan<R>::RTP;  // float2 per tile buffer
    static constexpr int NSLOT = FIRST ? 2 : 4;    // tiles x2, and their twiddles x2 after the first pass
    static constexpr size_t bytes = ((size_t)NSLOT * TS + RrPlan<R>::TW) * sizeof(float2);
};

template <int R, bool FIRST>
__global__ void __launch_bounds__(RrPlan<R>::NTR) k_fft_pass_rrdb(const __grid_constant__ PassArgs a, int tpc) {
    using P = RrPlan<R>;
    constexpr int A = P::A, B = P::B, C = P::C, RT = P::RT, RTP = P::RTP, NTR = P::NTR;
    constexpr int TS = RrdbPlan<R, FIRST>::TS;
    extern __shared__ float2 sm[];
    float2* twt = sm + RrdbPlan<R, FIRST>::NSLOT * TS;
    const int b = blockIdx.y;
    const int64_t ncol = a.M / R;
    const int64_t ntile = (ncol + RT - 1) / RT;
    const int64_t tile0 = (int64_t)blockIdx.x * tpc;
    const int64_t tile1 = min(ntile, tile0 + tpc);
    const float* sr = FIRST ? a.series + (int64_t)b * a.series_stride : nullptr;
    const float2* in = FIRST ? nullptr : a.in + (int64_t)b * a.in_stride;
    const int64_t nv = FIRST ? row_nv(a, b) : 0;
    // asynchronous copies of tile t (and its twiddles) into slot `slot`
    auto issue = [&](int64_t t, int slot) {
        float2* dst = sm + slot * TS;
        float2* dstw = sm + (2 + slot) * TS;
        const int64_t j0 = t * RT;
#pragma unroll 4
        for (int i = 0; i < (R * RT + NTR - 1) / NTR; ++i) {
            const int e = threadIdx.x + i * NTR;
            if ((R * RT) % NTR != 0 && e >= R * RT) break;
            const int jj = e % RT, r = e / RT;
            const int64_t j = j0 + jj;
            const int64_t n = j + (int64_t)r * ncol;
            if constexpr (FIRST) {
                // both samples, the first only (the odd tail), or none (zeros)
                const uint32_t nbytes = (j < ncol && 2 * n + 1 < nv) ? 8u : ((j < ncol && 2 * n < nv) ? 4u : 0u);
                cp_async8(dst + r * RTP + jj, nbytes ? (const void*)(sr + 2 * n) : (const void*)sr, nbytes);
            } else {
                const bool ok = j < ncol;
                cp_async8(dst + r * RTP + jj, ok ? (const void*)(in + n) : (const void*)in, ok ? 8u : 0u);
                const int64_t k = j & (a.Ns - 1);  // Ns: a power of two
                const bool okw = ok && k && r;     // the twiddle is used only there
                cp_async8(dstw + r * RTP + jj, okw ? (const void*)(a.ptw + (int64_t)r * a.Ns + k) : (const void*)a.ptw,
                          okw ? 8u : 0u);
            }
        }
    };
    issue(tile0, 0);
    cp_async_commit();
    // sub-stage twiddle tables from the global table exp(-2 pi i t / twM), once per CTA
    {
        const int64_t tstride = a.twM / R;
        int off = 0;
        if constexpr (B != 0) {
            for (int i = threadIdx.x; i < B * A; i += NTR) {
                const int q = i / A, k = i - q * A;
                twt[i] = a.tw[(int64_t)(q * k * (R / (B * A))) * tstride];
            }
            off = B * A;
        }
        for (int i = threadIdx.x; i < R; i += NTR) {
            const int q = i / (R / C), k = i - q * (R / C);
            twt[off + i] = a.tw[(int64_t)(q * k) * tstride];
        }
    }
    float mu_i = 0.f, mu_f = 0.f;
    if constexpr (FIRST) {
        __shared__ float s_mu[2];
        if (threadIdx.x == 0) {
            // mean = sum / N_v in FP64 (once per CTA), split as integer + fraction
            const double mu = (double)a.sums[b] / (double)nv;
            const double mi = rint(mu);
            s_mu[0] = (float)mi;
            s_mu[1] = (float)(mu - mi);
        }
        __syncthreads();
        mu_i = s_mu[0];
        mu_f = s_mu[1];
    }
    float2* o = a.out + (int64_t)b * a.out_stride;
    for (int64_t t = tile0; t < tile1; ++t) {
        const int slot = (int)((t - tile0) & 1);
        float2* buf = sm + slot * TS;
        const float2* wt = sm + (2 + slot) * TS;
        if (t + 1 < tile1) {
            issue(t + 1, slot ^ 1);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();  // tile t has landed (every thread's copies)
        const int64_t j0 = t * RT;
        // first sub-stage: radix A from the landed tile, ns = 1
        {
            constexpr int NB = R / A * RT;
            constexpr int PER = (NB + NTR - 1) / NTR;
            float2 x[PER][A];
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                const int e = threadIdx.x + p * NTR;
                if (NB % NTR == 0 || e < NB) {
                    const int jj = e % RT, bb = e / RT;
                    const int64_t j = j0 + jj;
#pragma unroll
                    for (int q = 0; q < A; ++q) {
                        const int r = bb + q * (R / A);
                        float2 v = make_float2(0.f, 0.f);
                        if (j < ncol) {
                            const float2 w = buf[r * RTP + jj];
                            if constexpr (FIRST) {
                                const int64_t n = j + (int64_t)r * ncol;
                                if (2 * n + 1 < nv) v = make_float2((w.x - mu_i) - mu_f, (w.y - mu_i) - mu_f);
                                else if (2 * n < nv) v.x = (w.x - mu_i) - mu_f;
                            } else {
                                v = w;
                                const int64_t k = j & (a.Ns - 1);
                                if (k && r) v = cmul(v, wt[r * RTP + jj]);
                            }
                        }
                        x[p][q] = v;
                    }
                    dft_any<A>(x[p]);
                }
            }
            __syncthreads();  // the tile is read: its buffer takes the sub-stage outputs
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                const int e = threadIdx.x + p * NTR;
                if (NB % NTR == 0 || e < NB) {
                    const int jj = e % RT, bb = e / RT;
#pragma unroll
                    for (int q = 0; q < A; ++q) buf[(bb * A + q) * RTP + jj] = x[p][q];
                }
            }
            __syncthreads();
        }
        if constexpr (B != 0) rr_mid<R, B, RT, NTR>(buf, twt, A);
        // last sub-stage: radix C, ns = R / C, straight to global memory (as k_fft_pass_rr)
        {
            constexpr int NS = R / C;
            const float2* tl = twt + (B ? B * A : 0);
            constexpr int NB = R / C * RT;
            constexpr int PER = (NB + NTR - 1) / NTR;
            const bool ns1 = a.Ns == 1;
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                const int e = threadIdx.x + p * NTR;
                if (NB % NTR == 0 || e < NB) {
                    const int jj = ns1 ? e / NS : e % RT;
                    const int bb = ns1 ? e % NS : e / RT;
                    float2 x[C];
#pragma unroll
                    for (int q = 0; q < C; ++q) {
                        x[q] = buf[(bb + q * NS) * RTP + jj];
                        if (q && bb) x[q] = cmul(x[q], tl[q * NS + bb]);
                    }
                    dft_any<C>(x);
                    const int64_t j = j0 + jj;
                    if (j < ncol) {
                        if (ns1) {
#pragma unroll
                            for (int q = 0; q < C; ++q) o[j * R + bb + q * NS] = x[q];
                        } else {
                            const int64_t kc = j & (a.Ns - 1);
                            float2* oo = o + (j / a.Ns) * a.Ns * R + kc;
#pragma unroll
                            for (int q = 0; q < C; ++q) oo[(int64_t)(bb + q * NS) * a.Ns] = x[q];
                        }
                    }
                }
            }
        }
        __syncthreads();  // the slot is free for the copies of tile t + 2
    }
}

// Staged tiles for the first pass up to radix 512 (PSS_FFT_STAGE_LATER=1: later passes up to
// radix 256 too); PSS_FFT_STAGE=0 keeps k_fft_pass_rr everywhere, PSS_FFT_STAGE_TPC sets the
// tiles per CTA (default 4)
int fft_stage_tpc() {
    static const int v = [] {
        const char* e = getenv("PSS_FFT_STAGE");
        if (e && e[0] == '0') return 0;
        const char* t = getenv("PSS_FFT_STAGE_TPC");
        const int x = t ? atoi(t) : 4;
        return x < 1 ? 1 : x;
    }();
    return v;
}

// PSS_FFT_RR=0 keeps the shared-memory sub-stage forms; by default the
// register-radix form runs.
bool fft_rr() {
    static const int v = [] {
        const char* e = getenv("PSS_FFT_RR");
        return e ? (e[0] == '1' ? 1 : 0) : 1;
    }();
    return v == 1;
}

template <int R>
cudaError_t run_pass_rr(const PassArgs& p, int nb, cudaStream_t s) {
    using P = RrPlan<R>;
    static_assert(P::A * (P::B ? P::B : 1) * P::C == R, "radix plan");
    const int tpc = fft_stage_tpc();
    // later passes stay unstaged by default: their four tile buffers (tiles and twiddles) leave
    // two CTAs per SM, slower than the unstaged pass (drift-scan FFT 1.33 against 1.46 ms staged)
    static const bool later = [] {
        const char* e = getenv("PSS_FFT_STAGE_LATER");
        return e && e[0] == '1';
    }();
    if constexpr (R <= 512) {
    if (tpc > 0 && (p.series ? R <= 512 : (later && R <= 256))) {
        const int64_t ntile = (p.M / R + P::RT - 1) / P::RT;
        const int per = (int)std::max<int64_t>(1, std::min<int64_t>(tpc, ntile));
        dim3 grid((unsigned)((ntile + per - 1) / per), (unsigned)nb);
        if (p.series) {
            constexpr size_t shm = RrdbPlan<R, true>::bytes;
            cudaError_t e = allow_smem((const void*)k_fft_pass_rrdb<R, true>, shm);
            if (e != cudaSuccess) return e;
            k_fft_pass_rrdb<R, true><<<grid, P::NTR, shm, s>>>(p, per);
        } else {
            constexpr size_t shm = RrdbPlan<R, false>::bytes;
            cudaError_t e = allow_smem((const void*)k_fft_pass_rrdb<R, false>, shm);
            if (e != cudaSuccess) return e;
            k_fft_pass_rrdb<R, false><<<grid, P::NTR, shm, s>>>(p, per);
        }
        return cudaGetLastError();
    }
    }
    const size_t shm = (size_t)(R * P::RTP + P::TW) * sizeof(float2);
    const void* k = p.series ? (const void*)k_fft_pass_rr<R, true> : (const void*)k_fft_pass_rr<R, false>;
    cudaError_t e = allow_smem(k, shm);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((p.M / R + P::RT - 1) / P::RT), (unsigned)nb);
    if (p.series) k_fft_pass_rr<R, true><<<grid, P::NTR, shm, s>>>(p);
    else k_fft_pass_rr<R, false><<<grid, P::NTR, shm, s>>>(p);
    return cudaGetLastError();
}

cudaError_t dispatch_pass(int R, const PassArgs& p, int nb, cudaStream_t s) {
    if (fft_rr()) {
        switch (R) {
            case 32: return run_pass_rr<32>(p, nb, s);
            case 64: return run_pass_rr<64>(p, nb, s);
            case 128: return run_pass_rr<128>(p, nb, s);
            case 256: return run_pass_rr<256>(p, nb, s);
            case 512: return run_pass_rr<512>(p, nb, s);
            case 1024: return run_pass_rr<1024>(p, nb, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (R) {
        case 32: return run_pass<32>(p, nb, s);
        case 64: return run_pass<64>(p, nb, s);
        case 128: return run_pass<128>(p, nb, s);
        case 256: return run_pass<256>(p, nb, s);
        case 512: return run_pass<512>(p, nb, s);
        case 1024: return run_pass<1024>(p, nb, s);
        default: return cudaErrorInvalidValue;
    }
}

__global__ void k_twiddles(float2* tw, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double s, c;
    sincospi(-2.0 * (double)t / (double)n, &s, &c);
    tw[t] = make_float2((float)c, (float)s);
}

// ---- real-to-complex post-processing + whitening ---------------------------
// One CTA per whitening block [bW, (b+1)W).  The lower median of |A_k|^2 is
// selected exactly on the float bit patterns (which order like the values for
// non-negative floats): a 2048-bin histogram of bits 30..20 locates the bin
// holding the wanted rank; the (few) values in that bin are gathered and the
// one of the right rank is found by counting, ties broken by position.  If
// that bin holds more than NCAND values, three further 8/8/4-bit histogram
// rounds on the remaining bits finish the selection instead.

template <int EPT>
__global__ void __launch_bounds__(256) k_r2c_whiten(const float2* Zall, int64_t z_stride, int64_t M, int W,
                                                    float2* out, int64_t out_stride, const float2* tw, int64_t twM,
                                                    int whiten, float* gains, int64_t gains_stride) {
    extern __shared__ uint32_t sh[];
    uint32_t* key = sh;              // [W]
    uint32_t* hist = sh + W;         // [NBIN]
    uint32_t* cand = hist + NBIN;    // [NCAND] values
    uint32_t* cpos = cand + NCAND;   // [NCAND] positions
    __shared__ uint32_t s_part[8], s_bin, s_rank, s_cnt, s_val;
    const int b = blockIdx.y;
    const int64_t k0 = (int64_t)blockIdx.x * W;
    const float2* Z = Zall + (int64_t)b * z_stride;
    float2* O = out + (int64_t)b * out_stride;
    const int nt = blockDim.x;
    const int64_t wstride = twM / (2 * M);  // exp(-2 pi i k / nfft)
    for (int i = threadIdx.x; i < NBIN; i += nt) hist[i] = 0u;
    if (threadIdx.x == 0) s_cnt = 0u;
    float2 A[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int64_t k = k0 + threadIdx.x + (int64_t)e * nt;
        const float2 zk = Z[k];
        const float2 zm = Z[(M - k) & (M - 1)];
        const float2 zc = make_float2(zm.x, -zm.y);
        const float2 sum = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
        const float2 dif = make_float2(0.5f * (zk.x - zc.x), 0.5f * (zk.y - zc.y));
        const float2 w = tw[k * wstride];
        const float2 wd = cmul(w, dif);
        float2 a = make_float2(sum.x + wd.y, sum.y - wd.x);  // sum - i * w * dif
        if (k == 0) a = make_float2(0.f, 0.f);
        A[e] = a;
        const float p = pow2(a);
        key[threadIdx.x + e * nt] = (k == 0) ? 0xFFFFFFFFu : __float_as_uint(p);
    }
    if (!whiten && !gains) {
#pragma unroll
        for (int e = 0; e < EPT; ++e) O[k0 + threadIdx.x + (int64_t)e * nt] = A[e];
        return;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const uint32_t kk = key[threadIdx.x + e * nt];
        if (kk != 0xFFFFFFFFu) atomicAdd(&hist[kk >> 20], 1u);
    }
    __syncthreads();
    const int m = (k0 == 0) ? W - 1 : W;
    const uint32_t rank0 = (uint32_t)((m - 1) / 2);
    // block scan over NBIN bins: thread t owns bins [t*BPT, (t+1)*BPT)
    const int BPT = NBIN / nt;
    {
        uint32_t tot = 0;
        // each thread starts at a different bin of its run so that a warp's reads fall in distinct banks
        const int rot = (int)threadIdx.x / (BPT >= 32 ? 1 : 32 / BPT);
        for (int i = 0; i < BPT; ++i) tot += hist[threadIdx.x * BPT + ((i + rot) & (BPT - 1))];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        uint32_t incl = tot;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31 || threadIdx.x == nt - 1) s_part[wid] = incl;
        __syncthreads();
        uint32_t before = incl - tot;
        for (int w2 = 0; w2 < wid; ++w2) before += s_part[w2];
        for (int i = 0; i < BPT; ++i) {
            const uint32_t c = hist[threadIdx.x * BPT + i];
            if (rank0 >= before && rank0 < before + c) {
                s_bin = (uint32_t)(threadIdx.x * BPT + i);
                s_rank = rank0 - before;
            }
            before += c;
        }
    }
    __syncthreads();
    const uint32_t bin = s_bin, rank = s_rank;
    const uint32_t nin = hist[bin];
    uint32_t med_bits;
    if (nin <= (uint32_t)NCAND) {
        // gather the bin's values, then count ranks (ties by position)
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int pos = threadIdx.x + e * nt;
            const uint32_t kk = key[pos];
            if (kk != 0xFFFFFFFFu && (kk >> 20) == bin) {
                const uint32_t slot = atomicAdd(&s_cnt, 1u);
                cand[slot] = kk;
                cpos[slot] = (uint32_t)pos;
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < nin; i += nt) {
            const uint32_t v = cand[i], pv = cpos[i];
            uint32_t r = 0;
            for (uint32_t q = 0; q < nin; ++q) {
                const uint32_t u = cand[q];
                r += (u < v) || (u == v && cpos[q] < pv);
            }
            if (r == rank) s_val = v;
        }
        __syncthreads();
        med_bits = s_val;
    } else {
        // many values share the top bits: finish with radix rounds on bits 19..0
        uint32_t prefix = bin << 20, mask = 0xFFF00000u, rk = rank;
        const int shifts[3] = {12, 4, 0};
        const int widths[3] = {8, 8, 4};
        for (int pass = 0; pass < 3; ++pass) {
            const int shift = shifts[pass];
            const uint32_t dmask = (1u << widths[pass]) - 1u;
            __syncthreads();
            for (int i = threadIdx.x; i < 256; i += nt) hist[i] = 0u;
            __syncthreads();
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                const uint32_t kk = key[threadIdx.x + e * nt];
                if (kk != 0xFFFFFFFFu && (kk & mask) == prefix) atomicAdd(&hist[(kk >> shift) & dmask], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t before = 0;
                for (uint32_t d = 0; d <= dmask; ++d) {
                    if (rk < before + hist[d]) {
                        s_bin = d;
                        s_rank = rk - before;
                        break;
                    }
                    before += hist[d];
                }
            }
            __syncthreads();
            prefix |= s_bin << shift;
            mask |= dmask << shift;
            rk = s_rank;
        }
        med_bits = prefix;
    }
    // scale sqrt(ln 2 / med) and gain ln 2 / med in FP64, once per CTA (FP64 is slow)
    __shared__ float s_scale;
    if (threadIdx.x == 0) {
        const float med = __uint_as_float(med_bits);
        const double g = med > 0.f ? 0.69314718055994530942 / (double)med : 0.0;
        s_scale = whiten ? (float)sqrt(g) : 1.f;
        if (gains) gains[(int64_t)b * gains_stride + blockIdx.x] = (float)g;
    }
    __syncthreads();
    const float scale = s_scale;
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int64_t k = k0 + threadIdx.x + (int64_t)e * nt;
        O[k] = make_float2(A[e].x * scale, A[e].y * scale);
    }
}

// ---- warp-per-block whitening (an alternative form for the autotuner) ------------
// The same R2C post-processing and exact lower median as k_r2c_whiten, with
// one warp per whitening block of W = 32 VPL bins: lane l holds bins
// k0 + l + 32 i (i < VPL) in registers and the selection uses a private
// shared-memory histogram of the warp, so no block-wide barrier is needed.
// Ties in the final rank are broken by position in the block, as there.
constexpr int WW = 4;  // warps per CTA

template <int VPL>
__global__ void __launch_bounds__(32 * WW) k_whiten_warp(const float2* Zall, int64_t z_stride, int64_t M,
                                                         float2* out, int64_t out_stride, const float2* tw,
                                                         int64_t twM, int whiten, float* gains,
                                                         int64_t gains_stride) {
    constexpr int W = 32 * VPL;
    __shared__ uint32_t s_hist[WW][NBIN];
    __shared__ uint32_t s_cand[WW][NCAND], s_cpos[WW][NCAND];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    const int64_t blk = (int64_t)blockIdx.x * WW + wq;
    if (blk >= M / W) return;
    const int b = blockIdx.y;
    const int64_t k0 = blk * W;
    const float2* Z = Zall + (int64_t)b * z_stride;
    float2* O = out + (int64_t)b * out_stride;
    const int64_t wstride = twM / (2 * M);  // exp(-2 pi i k / nfft)
    float2 A[VPL];
#pragma unroll
    for (int i = 0; i < VPL; ++i) {
        const int64_t k = k0 + lane + 32 * i;
        A[i] = r2c_bin(Z[k], Z[(M - k) & (M - 1)], tw[k * wstride], k);
    }
    if (!whiten && !gains) {
#pragma unroll
        for (int i = 0; i < VPL; ++i) O[k0 + lane + 32 * i] = A[i];
        return;
    }
    float* g = gains ? gains + (int64_t)b * gains_stride + blk : nullptr;
    whiten_block<VPL>(A, k0, lane, k0 == 0 ? W - 1 : W, s_hist[wq], s_cand[wq], s_cpos[wq], whiten, g, O + k0);
}

// Pairs of warps per block of W = 64 VPL bins (whiten_block_pair): half the
// registers per thread of the one-warp form, so twice the warps per SM.
constexpr int WP = 4;  // pairs per CTA

template <int VPL>
__global__ void __launch_bounds__(64 * WP, 4) k_whiten_pair(const float2* Zall, int64_t z_stride, int64_t M,
                                                        float2* out, int64_t out_stride, const float2* tw,
                                                        int64_t twM, int whiten, float* gains,
                                                        int64_t gains_stride) {
    constexpr int W = 64 * VPL;
    __shared__ uint32_t s_sh[WP][NBIN + 2 * NCAND + 8];
    const int lane = threadIdx.x & 31, pr = threadIdx.x >> 6, h = (threadIdx.x >> 5) & 1;
    const int64_t blk = (int64_t)blockIdx.x * WP + pr;
    if (blk >= M / W) return;  // both warps of a pair leave together
    const int b = blockIdx.y;
    const int64_t k0 = blk * W;
    const float2* Z = Zall + (int64_t)b * z_stride;
    float2* O = out + (int64_t)b * out_stride;
    const int64_t wstride = twM / (2 * M);  // exp(-2 pi i k / nfft)
    float2 A[VPL];
#pragma unroll
    for (int i = 0; i < VPL; ++i) {
        const int64_t k = k0 + h * 32 * VPL + lane + 32 * i;
        A[i] = r2c_bin(Z[k], Z[(M - k) & (M - 1)], tw[k * wstride], k);
    }
    if (!whiten && !gains) {
#pragma unroll
        for (int i = 0; i < VPL; ++i) O[k0 + h * 32 * VPL + lane + 32 * i] = A[i];
        return;
    }
    float* g = gains ? gains + (int64_t)b * gains_stride + blk : nullptr;
    whiten_block_pair<VPL>(A, k0, h, lane, k0 == 0 ? W - 1 : W, s_sh[pr], 1 + pr, whiten, g, O + k0);
}

// Whitening and the zmax 0 plane (the 32-tap half-bin interpolation of
// k_plane_z0) in one pass over the spectrum.  A CTA of WP warp pairs whitens
// WP consecutive blocks as k_whiten_pair does, stores each block's scale,
// puts the whitened bins of its range K0 .. K0 + WP W into shared memory
// (over the pairs' histograms, after a block barrier) and computes the plane
// values of its range whose windows (bins k - 15 .. k + 16) lie inside the
// range or reach past an end of the spectrum (zero there).  The 31 values
// whose windows cross an interior range boundary are left to k_z0_seams.
// Same operations in the same order as the whitening kernel followed by
// k_plane_z0 (bit-identical planes); the whitened spectrum never goes to HBM.
constexpr int Z0TAP = 32;              // 2m taps of the zmax 0 template
constexpr int Z0H = Z0TAP / 2 - 1;     // taps t = -Z0H .. Z0H + 1 around a bin
constexpr int Z0R = 8;                 // consecutive outputs per thread and round
constexpr int Z0S = Z0R == 16 ? 4 : 3; // one padding slot every 2^Z0S tile entries (conflict-free runs)
constexpr int SHW = NBIN + 2 * NCAND + 8;

template <int VPL>
__global__ void __launch_bounds__(64 * WP, 4) k_whiten_z0(const float2* Zall, int64_t z_stride, int64_t M,
                                                      float* plane, int64_t plane_stride, const float2* tw,
                                                      int64_t twM, const float* tap_scale1, float* wscale) {
    constexpr int W = 64 * VPL;
    constexpr int KB = WP * W;            // bins per CTA
    constexpr int TW = KB + Z0TAP - 1;     // tile: bins K0 - Z0H .. K0 + KB + Z0H
    constexpr int TWP = TW + (TW >> Z0S) + 1;
    constexpr int NTH = 64 * WP;
    static_assert(2 * TWP <= WP * SHW, "the tile fits in the pairs' whitening scratch");
    static_assert(KB % Z0R == 0, "whole runs of outputs");
    __shared__ __align__(16) uint32_t s_raw[WP * SHW];
    const int lane = threadIdx.x & 31, pr = threadIdx.x >> 6, h = (threadIdx.x >> 5) & 1;
    const int64_t nblk = M / W;
    const int64_t blk = (int64_t)blockIdx.x * WP + pr;
    const bool have = blk < nblk;
    const int b = blockIdx.y;
    const int64_t k0 = blk * W;
    const int64_t K0 = (int64_t)blockIdx.x * KB;
    const float2* Z = Zall + (int64_t)b * z_stride;
    const int64_t wstride = twM / (2 * M);  // exp(-2 pi i k / nfft)
    float2 A[VPL];
    if (have) {
#pragma unroll
        for (int i = 0; i < VPL; ++i) {
            const int64_t k = k0 + h * 32 * VPL + lane + 32 * i;
            A[i] = r2c_bin(Z[k], Z[(M - k) & (M - 1)], tw[k * wstride], k);
        }
        const float scale = whiten_block_pair<VPL>(A, k0, h, lane, k0 == 0 ? W - 1 : W, s_raw + pr * SHW, 1 + pr, 1,
                                                   nullptr, nullptr);
        if (h == 0 && lane == 0) wscale[(int64_t)b * nblk + blk] = scale;
    }
    __syncthreads();  // every pair is done with its histogram
    float2* tile = reinterpret_cast<float2*>(s_raw);
    if (have) {
#pragma unroll
        for (int i = 0; i < VPL; ++i) {
            const int u = (int)(k0 - K0) + h * 32 * VPL + lane + 32 * i + Z0H;
            tile[u + (u >> Z0S)] = A[i];
        }
    }
    for (int u = threadIdx.x; u < TW; u += NTH) {
        const int64_t k = K0 - Z0H + u;
        if (k < K0 || k >= K0 + KB || k >= M) tile[u + (u >> Z0S)] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float s1 = *tap_scale1;
    float2* P = reinterpret_cast<float2*>(plane + (int64_t)b * plane_stride);
    // outputs whose windows cross an interior boundary of the CTA ranges
    const int64_t lo_ok = K0 > 0 ? K0 + Z0H : K0;
    const int64_t hi_ok = K0 + KB < M ? K0 + KB - Z0H - 1 : M;
#pragma unroll 1
    for (int ub = (int)threadIdx.x * Z0R; ub < KB; ub += NTH * Z0R) {  // ub: tile index of the first window
        float re[Z0R], im[Z0R], p0[Z0R];
#pragma unroll
        for (int i = 0; i < Z0R; ++i) re[i] = im[i] = p0[i] = 0.f;
        const float2* w = tile + ub + (ub >> Z0S);
#pragma unroll
        for (int j = 0; j < Z0R + Z0TAP - 1; ++j) {
            const float2 x = w[j + (j >> Z0S)];
#pragma unroll
            for (int i = 0; i < Z0R; ++i) {
                const int ti = j - i;
                if (ti >= 0 && ti < Z0TAP) {
                    re[i] = fmaf(x.x, z0_tap<Z0TAP>(ti), re[i]);
                    im[i] = fmaf(x.y, z0_tap<Z0TAP>(ti), im[i]);
                }
                if (ti == Z0H) p0[i] = pow2(x);
            }
        }
        const int64_t kb = K0 + ub;
#pragma unroll
        for (int i = 0; i < Z0R; ++i) {
            const int64_t k = kb + i;
            const float r = re[i] * s1, q = im[i] * s1;
            if (k >= lo_ok && k < hi_ok) P[k] = make_float2(p0[i], pow2(r, q));
        }
    }
}

// The plane values next to the interior boundaries K = c KB (0 < K < M) of
// k_whiten_z0's ranges: outputs K - Z0H - 1 .. K + Z0H - 1, one warp per
// boundary, from the bins K - 2 Z0H - 1 .. K + 2 Z0H re-derived from the half
// spectrum (r2c_bin) times their blocks' scales.  Same arithmetic and order
// as k_plane_z0.
constexpr int SEAM_WARPS = 4;

__global__ void __launch_bounds__(32 * SEAM_WARPS) k_z0_seams(const float2* Zall, int64_t z_stride, int64_t M, int W,
                                                              int KB, float* plane, int64_t plane_stride,
                                                              const float2* tw, int64_t twM, const float* tap_scale1,
                                                              const float* wscale) {
    constexpr int NW = 2 * Z0TAP - 2;  // bins of the 2 Z0H + 1 windows
    __shared__ float2 win[SEAM_WARPS][NW];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t K = ((int64_t)blockIdx.x * SEAM_WARPS + warp + 1) * KB;
    if (K >= M) return;  // no block barrier below
    const int b = blockIdx.y;
    const float2* Z = Zall + (int64_t)b * z_stride;
    const float* sc = wscale + (int64_t)b * (M / W);
    const int64_t wstride = twM / (2 * M);
    const int64_t kw = K - 2 * Z0H - 1;  // first bin of the windows (>= 1: K >= KB >= 256)
    for (int j = lane; j < NW; j += 32) {
        const int64_t k = kw + j;
        const float2 a = r2c_bin(Z[k], Z[(M - k) & (M - 1)], tw[k * wstride], k);
        const float s = sc[k / W];
        win[warp][j] = make_float2(a.x * s, a.y * s);
    }
    __syncwarp();
    if (lane >= 2 * Z0H + 1) return;
    float re = 0.f, im = 0.f, p0 = 0.f;
#pragma unroll
    for (int ti = 0; ti < Z0TAP; ++ti) {
        const float2 x = win[warp][lane + ti];
        re = fmaf(x.x, z0_tap<Z0TAP>(ti), re);
        im = fmaf(x.y, z0_tap<Z0TAP>(ti), im);
        if (ti == Z0H) p0 = pow2(x);
    }
    const float s1 = *tap_scale1;
    const float r = re * s1, q = im * s1;
    reinterpret_cast<float2*>(plane + (int64_t)b * plane_stride)[K - Z0H - 1 + lane] = make_float2(p0, pow2(r, q));
}

// Pass radices of an M-point FFT, M = 2^L: the fewest passes of radix
// 2^5 .. 2^10 (ceil(L / 10)); variant 0 splits L evenly, larger parts
// first; variants 1.. are the other splits of L into that many parts within
// [5, 10] (used by the autotuner).  Returns false past the last variant.
bool radix_variant(int64_t M, int variant, int* rad, int* np) {
    int L = 0;
    while ((int64_t(1) << L) < M) ++L;
    int p = (L + 9) / 10;
    if (p < 1) p = 1;
    int parts[4];
    for (int i = 0; i < p; ++i) parts[i] = L / p + (i < L % p ? 1 : 0);
    int v = 0;
    if (variant > 0) {
        // enumerate compositions of L into p parts in [5, 10], skipping the even split
        int c[4] = {5, 5, 5, 5};
        bool found = false;
        while (!found) {
            int sum = 0;
            for (int i = 0; i < p; ++i) sum += c[i];
            bool even = true;
            for (int i = 0; i < p; ++i) even &= (c[i] == parts[i]);
            if (sum == L && !even && ++v == variant) {
                for (int i = 0; i < p; ++i) parts[i] = c[i];
                found = true;
                break;
            }
            int i = p - 1;
            while (i >= 0 && c[i] == 10) c[i--] = 5;
            if (i < 0) return false;
            ++c[i];
        }
    }
    for (int i = 0; i < p; ++i) rad[i] = 1 << parts[i];
    *np = p;
    return true;
}

}  // namespace

int fft_pass_plan(int64_t M, int variant, int* rad) {
    int np = 0;
    if (!radix_variant(M, variant, rad, &np)) return 0;
    return np;
}

namespace {
// inter-pass twiddles of a later pass: out[r Ns + k] = tw[r k twM / (Ns R)]
__global__ void k_pass_twiddles(float2* out, const float2* tw, int64_t twM, int R, int64_t Ns) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)R * Ns) return;
    const int64_t r = i / Ns, k = i - r * Ns;
    out[i] = tw[r * k * (twM / (Ns * R))];
}
}  // namespace

cudaError_t launch_pass_twiddles(float2* out, const float2* tw, int64_t twM, int R, int64_t Ns, cudaStream_t s) {
    const int64_t n = (int64_t)R * Ns;
    k_pass_twiddles<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, tw, twM, R, Ns);
    return cudaGetLastError();
}

cudaError_t launch_twiddles(float2* tw, int64_t n, cudaStream_t s) {
    k_twiddles<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tw, n);
    return cudaGetLastError();
}

cudaError_t launch_fft_whiten(const FftArgs& a, cudaStream_t s, Ctx* prof_ctx) {
    const int64_t M = a.nfft / 2;
    if (M < 64 || (M & (M - 1)) != 0) return cudaErrorInvalidValue;
    if (!a.tw || a.twM < a.nfft || a.twM % a.nfft) return cudaErrorInvalidValue;
    int rad[4], np = 0;
    if (!radix_variant(M, a.fft_variant, rad, &np)) return cudaErrorInvalidValue;
    for (int i = 0; i < np; ++i)
        if (rad[i] < 32 || rad[i] > 1024) return cudaErrorInvalidValue;
    PassArgs p{};
    p.M = M;
    p.nv = a.nv;
    p.nv_rows = a.nv_rows;
    p.sums = a.sums;
    p.tw = a.tw;
    p.twM = a.twM;
    int64_t Ns = 1;
    const float2* in = nullptr;
    float2* bufs[2] = {a.bufA, a.bufB};
    float2* cur = nullptr;
    for (int i = 0; i < np; ++i) {
        p.in = in;
        p.in_stride = M;
        p.series = (i == 0) ? a.series : nullptr;
        p.series_stride = a.series_stride;
        cur = bufs[i & 1];
        p.out = cur;
        p.out_stride = M;
        p.Ns = Ns;
        p.ptw = a.ptw[i];
        if (i > 0 && !p.ptw) return cudaErrorInvalidValue;
        ProfScope ps(prof_ctx, 2, s);
        cudaError_t e = dispatch_pass(rad[i], p, a.nb, s);
        if (e != cudaSuccess) return e;
        in = cur;
        Ns *= rad[i];
    }
    const int W = a.whiten_block;
    if (W < 64 || W > 4096 || (W & (W - 1)) != 0 || M % W != 0) return cudaErrorInvalidValue;
    if (a.z0_plane && a.whiten && !a.gains_out && (W == 1024 || W == 512 || W == 256)) {
        // whitening + zmax 0 plane, then the values at the CTA range boundaries
        if (!a.z0_scale1 || !a.wscale) return cudaErrorInvalidValue;
        const int KB = WP * W;
        dim3 g2((unsigned)((M / W + WP - 1) / WP), (unsigned)a.nb);
        // both kernels are profiled as the whitening stage (the plane stage then has no launches)
        ProfScope ps(prof_ctx, 3, s);
        {
            if (W == 1024)
                k_whiten_z0<16><<<g2, 64 * WP, 0, s>>>(in, M, M, a.z0_plane, a.z0_plane_stride, a.tw, a.twM,
                                                       a.z0_scale1, a.wscale);
            else if (W == 512)
                k_whiten_z0<8><<<g2, 64 * WP, 0, s>>>(in, M, M, a.z0_plane, a.z0_plane_stride, a.tw, a.twM,
                                                      a.z0_scale1, a.wscale);
            else
                k_whiten_z0<4><<<g2, 64 * WP, 0, s>>>(in, M, M, a.z0_plane, a.z0_plane_stride, a.tw, a.twM,
                                                      a.z0_scale1, a.wscale);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        const int64_t nseam = (M - 1) / KB;  // boundaries K = c KB, 0 < K < M
        if (nseam > 0) {
            dim3 g3((unsigned)((nseam + SEAM_WARPS - 1) / SEAM_WARPS), (unsigned)a.nb);
            k_z0_seams<<<g3, 32 * SEAM_WARPS, 0, s>>>(in, M, M, W, KB, a.z0_plane, a.z0_plane_stride, a.tw, a.twM,
                                                      a.z0_scale1, a.wscale);
        }
        return cudaGetLastError();
    }
    if (a.whiten_form == 2 && (W == 1024 || W == 512 || W == 256)) {
        dim3 g2((unsigned)((M / W + WP - 1) / WP), (unsigned)a.nb);
        ProfScope ps(prof_ctx, 3, s);
        if (W == 1024)
            k_whiten_pair<16><<<g2, 64 * WP, 0, s>>>(in, M, M, a.spec_out, a.spec_stride, a.tw, a.twM, a.whiten,
                                                     a.gains_out, a.gains_stride);
        else if (W == 512)
            k_whiten_pair<8><<<g2, 64 * WP, 0, s>>>(in, M, M, a.spec_out, a.spec_stride, a.tw, a.twM, a.whiten,
                                                    a.gains_out, a.gains_stride);
        else
            k_whiten_pair<4><<<g2, 64 * WP, 0, s>>>(in, M, M, a.spec_out, a.spec_stride, a.tw, a.twM, a.whiten,
                                                    a.gains_out, a.gains_stride);
        return cudaGetLastError();
    }
    if (a.whiten_form == 1 && (W == 1024 || W == 512 || W == 256)) {
        dim3 g2((unsigned)((M / W + WW - 1) / WW), (unsigned)a.nb);
        ProfScope ps(prof_ctx, 3, s);
        if (W == 1024)
            k_whiten_warp<32><<<g2, 32 * WW, 0, s>>>(in, M, M, a.spec_out, a.spec_stride, a.tw, a.twM, a.whiten,
                                                     a.gains_out, a.gains_stride);
        else if (W == 512)
            k_whiten_warp<16><<<g2, 32 * WW, 0, s>>>(in, M, M, a.spec_out, a.spec_stride, a.tw, a.twM, a.whiten,
                                                     a.gains_out, a.gains_stride);
        else
            k_whiten_warp<8><<<g2, 32 * WW, 0, s>>>(in, M, M, a.spec_out, a.spec_stride, a.tw, a.twM, a.whiten,
                                                    a.gains_out, a.gains_stride);
        return cudaGetLastError();
    }
    const int nt = W < 256 ? W : 256;
    const size_t shm = (size_t)(W + NBIN + 2 * NCAND) * sizeof(uint32_t);
    dim3 grid((unsigned)(M / W), (unsigned)a.nb);
    ProfScope ps(prof_ctx, 3, s);
    switch (W / nt) {
#define PSS_WHITEN(E)                                                                                       \
    case E: {                                                                                               \
        cudaError_t e = allow_smem((const void*)k_r2c_whiten<E>, shm);                               \
        if (e != cudaSuccess) return e;                                                                     \
        k_r2c_whiten<E><<<grid, nt, shm, s>>>(in, M, M, W, a.spec_out, a.spec_stride, a.tw, a.twM, a.whiten, \
                                              a.gains_out, a.gains_stride);                                 \
        break;                                                                                              \
    }
        PSS_WHITEN(1)
        PSS_WHITEN(2)
        PSS_WHITEN(4)
        PSS_WHITEN(8)
        PSS_WHITEN(16)
#undef PSS_WHITEN
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pss
