// Batched real FFT of the dedispersed series and block-median whitening
// (paper Sect. 2 step 3, realfft; whitening is not described in the paper).
//
// A real series y of length nfft is packed as z[n] = y[2n] + i y[2n+1] and
// transformed with an M = nfft/2 point complex FFT; the half spectrum
//   A_k = (Z_k + conj Z_{M-k}) / 2 - (i/2) e^{-2 pi i k / nfft} (Z_k - conj Z_{M-k})
// is formed in the whitening kernel.
//
// The complex FFT is a Stockham auto-sort FFT with a few large-radix passes
// (radix R = 64..1024, product = M).  In the pass with running length Ns,
// element j + r*M/R (r < R) of each of M/R columns is multiplied by
// exp(-2 pi i r (j mod Ns) / (Ns R)), transformed by an R-point DFT and
// written to (j / Ns) * Ns * R + (j mod Ns) + r * Ns.  A CTA owns TJ = 8
// consecutive columns, reads them with contiguous 64-byte rows, does the
// R-point DFT in shared memory with radix-4 (and one radix-2) Stockham
// sub-stages, and writes contiguous rows.  Two passes cover M <= 2^20.
//
// The first pass also subtracts the series mean (exact integer sum / N_v,
// split into an integer and a fractional part so the FP32 subtraction is
// exact up to one rounding) and zero-pads past N_v.
#include <math.h>

#include "pss_internal.h"

namespace pss {

namespace {

constexpr int TJ = 8;       // columns per CTA
constexpr int TJP = TJ + 1; // padded shared-memory row (bank spread)
constexpr int NT = 256;     // threads per CTA

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

// exp(-2 pi i num / den) for integers 0 <= num < den, den a power of two
__device__ __forceinline__ float2 twiddle(int64_t num, int64_t den) {
    float s, c;
    sincospif(-2.0f * (float)num / (float)den, &s, &c);
    return make_float2(c, s);
}

// In-place R-point DFT of TJ columns held in shared memory as
// buf[r * TJP + jj], by Stockham sub-stages of radix 4 (and one of radix 2
// when log2 R is odd).
template <int R>
__device__ void smem_dft(float2* buf) {
    constexpr int LOG = (R == 32) ? 5 : (R == 64) ? 6 : (R == 128) ? 7 : (R == 256) ? 8 : (R == 512) ? 9 : 10;
    int ns = 1;
    if (LOG & 1) {
        // radix-2 sub-stage first
        constexpr int NB = R / 2 * TJ;
        constexpr int PER = (NB + NT - 1) / NT;
        float2 v[PER][2];
        int dst[PER];
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int e = threadIdx.x + p * NT;
            if (e < NB) {
                const int jj = e % TJ, b = e / TJ;
                v[p][0] = buf[b * TJP + jj];
                v[p][1] = buf[(b + R / 2) * TJP + jj];
                dst[p] = (2 * b) * TJP + jj;  // ns = 1: idxD = 2b
            }
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int e = threadIdx.x + p * NT;
            if (e < NB) {
                buf[dst[p]] = cadd(v[p][0], v[p][1]);
                buf[dst[p] + TJP] = csub(v[p][0], v[p][1]);
            }
        }
        __syncthreads();
        ns = 2;
    }
    for (; ns < R; ns *= 4) {
        constexpr int NB = R / 4 * TJ;
        constexpr int PER = (NB + NT - 1) / NT;
        float2 v[PER][4];
        int dst[PER];
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int e = threadIdx.x + p * NT;
            if (e < NB) {
                const int jj = e % TJ, b = e / TJ;
                const int k = b % ns;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float2 x = buf[(b + q * (R / 4)) * TJP + jj];
                    if (q && k) x = cmul(x, twiddle((int64_t)q * k, 4 * ns));
                    v[p][q] = x;
                }
                dst[p] = ((b / ns) * ns * 4 + k) * TJP + jj;
            }
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < PER; ++p) {
            const int e = threadIdx.x + p * NT;
            if (e < NB) {
                const float2 a0 = v[p][0], a1 = v[p][1], a2 = v[p][2], a3 = v[p][3];
                const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
                const float2 s13 = cadd(a1, a3), d13 = mul_mi(csub(a1, a3));
                buf[dst[p]] = cadd(s02, s13);
                buf[dst[p] + ns * TJP] = cadd(d02, d13);
                buf[dst[p] + 2 * ns * TJP] = csub(s02, s13);
                buf[dst[p] + 3 * ns * TJP] = csub(d02, d13);
            }
        }
        __syncthreads();
    }
}

struct PassArgs {
    const float2* in;          // [nb][in_stride] complex (null on the first pass)
    int64_t in_stride;
    const float* series;       // first pass: real series [nb][series_stride]
    int64_t series_stride;
    const unsigned long long* sums;
    int64_t nv;
    float2* out;
    int64_t out_stride;
    int64_t M;
    int64_t Ns;
};

template <int R>
__global__ void __launch_bounds__(NT) k_fft_pass(PassArgs a) {
    extern __shared__ float2 buf[];
    const int b = blockIdx.y;
    const int64_t ncol = a.M / R;
    const int64_t j0 = (int64_t)blockIdx.x * TJ;
    const bool first = (a.series != nullptr);

    float mu_i = 0.f, mu_f = 0.f;
    if (first) {
        // mean = sum / N_v in FP64, split as integer + fraction
        const double mu = (double)a.sums[b] / (double)a.nv;
        const double mi = rint(mu);
        mu_i = (float)mi;
        mu_f = (float)(mu - mi);
    }
    // load with twiddles
    for (int e = threadIdx.x; e < R * TJ; e += NT) {
        const int jj = e % TJ, r = e / TJ;
        const int64_t j = j0 + jj;
        float2 x = make_float2(0.f, 0.f);
        if (j < ncol) {
            const int64_t n = j + (int64_t)r * ncol;
            if (first) {
                const float* s = a.series + (int64_t)b * a.series_stride;
                const int64_t m0 = 2 * n, m1 = 2 * n + 1;
                x.x = (m0 < a.nv) ? (s[m0] - mu_i) - mu_f : 0.f;
                x.y = (m1 < a.nv) ? (s[m1] - mu_i) - mu_f : 0.f;
            } else {
                x = a.in[(int64_t)b * a.in_stride + n];
                const int64_t k = j % a.Ns;
                if (k && r) x = cmul(x, twiddle(((int64_t)r * k) % (a.Ns * R), a.Ns * R));
            }
        }
        buf[r * TJP + jj] = x;
    }
    __syncthreads();
    smem_dft<R>(buf);
    // store
    float2* o = a.out + (int64_t)b * a.out_stride;
    if (a.Ns == 1) {
        for (int e = threadIdx.x; e < R * TJ; e += NT) {
            const int r = e % R, jj = e / R;
            const int64_t j = j0 + jj;
            if (j < ncol) o[j * R + r] = buf[r * TJP + jj];
        }
    } else {
        for (int e = threadIdx.x; e < R * TJ; e += NT) {
            const int jj = e % TJ, r = e / TJ;
            const int64_t j = j0 + jj;
            if (j < ncol) {
                const int64_t k = j % a.Ns;
                o[(j / a.Ns) * a.Ns * R + k + (int64_t)r * a.Ns] = buf[r * TJP + jj];
            }
        }
    }
}

template <int R>
cudaError_t run_pass(const PassArgs& p, int nb, cudaStream_t s) {
    const size_t shm = (size_t)R * TJP * sizeof(float2);
    cudaFuncSetAttribute(k_fft_pass<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    dim3 grid((unsigned)((p.M / R + TJ - 1) / TJ), (unsigned)nb);
    k_fft_pass<R><<<grid, NT, shm, s>>>(p);
    return cudaGetLastError();
}

cudaError_t dispatch_pass(int R, const PassArgs& p, int nb, cudaStream_t s) {
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

// ---- real-to-complex post-processing + whitening ---------------------------
// One CTA per whitening block [bW, (b+1)W).  The lower median of |A_k|^2 is
// found exactly by a 4-digit radix select on the float bit patterns (which
// order like the values for non-negative floats).
template <int EPT>
__global__ void __launch_bounds__(256) k_r2c_whiten(const float2* Zall, int64_t z_stride, int64_t M,
                                                    int W, float2* out, int64_t out_stride) {
    extern __shared__ uint32_t sh[];
    uint32_t* key = sh;             // [W]
    uint32_t* hist = sh + W;        // [256]
    __shared__ uint32_t s_digit, s_rank;
    const int b = blockIdx.y;
    const int64_t k0 = (int64_t)blockIdx.x * W;
    const float2* Z = Zall + (int64_t)b * z_stride;
    float2* O = out + (int64_t)b * out_stride;
    float2 A[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int64_t k = k0 + threadIdx.x + (int64_t)e * blockDim.x;
        const float2 zk = Z[k];
        const float2 zm = Z[(M - k) & (M - 1)];
        const float2 zc = make_float2(zm.x, -zm.y);
        const float2 sum = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
        const float2 dif = make_float2(0.5f * (zk.x - zc.x), 0.5f * (zk.y - zc.y));
        // -(i) * w * dif,  w = exp(-2 pi i k / nfft) = exp(-pi i k / M)
        float s, c;
        sincospif(-(float)k / (float)M, &s, &c);
        const float2 wd = make_float2(c * dif.x - s * dif.y, c * dif.y + s * dif.x);
        float2 a = make_float2(sum.x + wd.y, sum.y - wd.x);
        if (k == 0) a = make_float2(0.f, 0.f);
        A[e] = a;
        const float p = a.x * a.x + a.y * a.y;
        key[threadIdx.x + e * blockDim.x] = (k == 0) ? 0xFFFFFFFFu : __float_as_uint(p);
    }
    const int m = (k0 == 0) ? W - 1 : W;
    uint32_t rank = (uint32_t)((m - 1) / 2);
    uint32_t prefix = 0u, mask = 0u;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0u;
        __syncthreads();
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const uint32_t kk = key[threadIdx.x + e * blockDim.x];
            if (kk != 0xFFFFFFFFu && (kk & mask) == prefix) atomicAdd(&hist[(kk >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            // warp 0 scans the 256 bins (8 per lane) to find the digit
            const int lane = threadIdx.x;
            uint32_t loc[8], tot = 0;
            for (int i = 0; i < 8; ++i) {
                loc[i] = hist[lane * 8 + i];
                tot += loc[i];
            }
            uint32_t incl = tot;
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            uint32_t before = incl - tot;
            for (int i = 0; i < 8; ++i) {
                if (rank >= before && rank < before + loc[i]) {
                    s_digit = (uint32_t)(lane * 8 + i);
                    s_rank = rank - before;
                }
                before += loc[i];
            }
        }
        __syncthreads();
        prefix |= s_digit << shift;
        mask |= 255u << shift;
        rank = s_rank;
        __syncthreads();
    }
    const float med = __uint_as_float(prefix);
    float scale = 0.f;
    if (med > 0.f) scale = (float)sqrt(0.69314718055994530942 / (double)med);
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
        const int64_t k = k0 + threadIdx.x + (int64_t)e * blockDim.x;
        O[k] = make_float2(A[e].x * scale, A[e].y * scale);
    }
}

void radix_plan(int64_t M, int* rad, int* np) {
    int L = 0;
    while ((int64_t(1) << L) < M) ++L;
    int p = (L + 9) / 10;
    if (p < 1) p = 1;
    // split L into p parts, larger ones first
    for (int i = 0; i < p; ++i) {
        int li = L / p + (i < L % p ? 1 : 0);
        rad[i] = 1 << li;
    }
    *np = p;
}

}  // namespace

cudaError_t launch_fft_whiten(const FftArgs& a, cudaStream_t s, Ctx* prof_ctx) {
    const int64_t M = a.nfft / 2;
    if (M < 64 || (M & (M - 1)) != 0) return cudaErrorInvalidValue;
    int rad[4], np = 0;
    radix_plan(M, rad, &np);
    for (int i = 0; i < np; ++i)
        if (rad[i] < 32 || rad[i] > 1024) return cudaErrorInvalidValue;
    PassArgs p{};
    p.M = M;
    p.nv = a.nv;
    p.sums = a.sums;
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
        ProfScope ps(prof_ctx, 2, s);
        cudaError_t e = dispatch_pass(rad[i], p, a.nb, s);
        if (e != cudaSuccess) return e;
        in = cur;
        Ns *= rad[i];
    }
    const int W = a.whiten_block;
    if (W < 64 || W > 4096 || (W & (W - 1)) != 0 || M % W != 0) return cudaErrorInvalidValue;
    const int nt = W < 256 ? W : 256;
    const size_t shm = (size_t)(W + 256) * sizeof(uint32_t);
    dim3 grid((unsigned)(M / W), (unsigned)a.nb);
    ProfScope ps(prof_ctx, 3, s);
    switch (W / nt) {
#define PSS_WHITEN(E)                                                                            \
    case E:                                                                                      \
        cudaFuncSetAttribute(k_r2c_whiten<E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm); \
        k_r2c_whiten<E><<<grid, nt, shm, s>>>(in, M, M, W, a.spec_out, a.spec_stride);           \
        break;
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
