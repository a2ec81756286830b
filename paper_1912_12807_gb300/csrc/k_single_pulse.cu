// Single-pulse (boxcar matched-filter) search of dedispersed series: the
// step after dedispersion in the paper's pipeline (single_pulse_search.py,
// Sect. 2 step 7; long-period pulsars are found this way, Sect. 5.3).
//
// Per trial: mu = S1/N and sigma = sqrt((S2 - S1*S1/N)/N) from the exact
// integer moments S1 = sum s, S2 = sum s^2; for each boxcar width w,
// B_w[t] = sum_{k<w} s[t+k] (exact, t <= N - w) is a detection when
// B_w[t] >= w*mu + thr*sigma*sqrt(w) and it is a local maximum over its
// own width (strictly above the w - 1 values before it, not below the
// w - 1 after it).  The FP64 arithmetic is written with round-to-nearest
// intrinsics in the stated order so that no multiply-add is contracted and
// the threshold is the same number the host computes.
//
// k_sp_moments: one pass over the series, 64-bit integer sums.
// k_sp_thresholds: the integer threshold of every (trial, width), FP64.
// k_sp_detect: a CTA owns TS samples of one trial; it stages the samples
// [t0 - wmax + 1, t0 + TS + 2 wmax - 2] in shared memory as a prefix sum
// (32-bit when every sum of the tile fits, else 64-bit) (so every B_w the tile and its local-maximum windows need is
// one subtraction), then tests every (t, w).  Detections are appended
// with an atomic counter; past `cap` they are only counted.
#include <limits.h>

#include "pss_internal.h"

namespace pss {

namespace {

constexpr int TS = 2048;  // samples per CTA
constexpr int NT = 256;

__global__ void __launch_bounds__(NT) k_sp_moments(const int32_t* __restrict__ series, int64_t stride, int64_t n,
                                                   unsigned long long* s1, unsigned long long* s2) {
    const int b = blockIdx.y;
    const int32_t* s = series + (int64_t)b * stride;
    unsigned long long a1 = 0ull, a2 = 0ull;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        const unsigned long long v = (unsigned long long)(uint32_t)s[i];
        a1 += v;
        a2 += v * v;
    }
    for (int off = 16; off > 0; off >>= 1) {
        a1 += __shfl_xor_sync(0xffffffffu, a1, off);
        a2 += __shfl_xor_sync(0xffffffffu, a2, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(s1 + b, a1);
        atomicAdd(s2 + b, a2);
    }
}

// One thread per (trial, width): the integer threshold ceil(w*mu +
// thr*sigma*sqrt(w)) (B is an integer below 2^53, exact as a double, so
// (double)B >= thr exactly when B >= ceil(thr)); LLONG_MAX when sigma is 0.
__global__ void k_sp_thresholds(const __grid_constant__ SpArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nb * a.nw) return;
    const int b = i / a.nw, wi = i - b * a.nw;
    const double fS1 = (double)a.s1[b], fS2 = (double)a.s2[b], fN = (double)a.n;
    const double mu = __ddiv_rn(fS1, fN);
    double var = __ddiv_rn(__dsub_rn(fS2, __ddiv_rn(__dmul_rn(fS1, fS1), fN)), fN);
    if (!(var > 0.0)) var = 0.0;
    const double sigma = __dsqrt_rn(var);
    long long t = LLONG_MAX;
    if (sigma > 0.0) {
        const double w = (double)a.w[wi];
        const double thr = __dadd_rn(__dmul_rn(w, mu), __dmul_rn(__dmul_rn(a.thr, sigma), __dsqrt_rn(w)));
        const double c = ceil(thr);
        t = c > 9.0e18 ? LLONG_MAX : (c < -9.0e18 ? LLONG_MIN : (long long)c);
    }
    a.thr_tab[i] = t;
}

// T: the prefix-sum type; 32-bit when every window sum of the launch fits
// (the host checks the bound), else 64-bit.
template <typename T>
__global__ void __launch_bounds__(NT) k_sp_detect(const __grid_constant__ SpArgs a) {
    extern __shared__ __align__(16) unsigned char sp_raw[];
    T* R = reinterpret_cast<T*>(sp_raw);  // prefix sums relative to `base`
    __shared__ T s_tot[NT];
    const int b = blockIdx.y;
    const int64_t n = a.n;
    const int64_t t0 = (int64_t)blockIdx.x * TS;
    const int32_t* s = a.series + (int64_t)b * a.stride;
    const long long* thr_b = a.thr_tab + (int64_t)b * a.nw;
    if (thr_b[0] == LLONG_MAX) return;  // sigma 0: no detections (uniform over the CTA)
    const int64_t base = max((int64_t)0, t0 - a.wmax + 1);
    const int64_t last = min(n, t0 + TS + 2 * (int64_t)a.wmax - 2);  // largest prefix index needed
    const int L = (int)(last - base + 1);                           // R[0 .. L-1]
    // R[k] = sum_{base <= j < base + k} s[j]: per-thread segment sums, then a scan
    const int seg = (L + NT - 1) / NT;
    const int k0 = threadIdx.x * seg;
    T acc = 0;
    for (int k = k0; k < min(k0 + seg, L - 1); ++k) acc += s[base + k];
    s_tot[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        // exclusive scan of the NT segment totals by one warp (8 per lane)
        constexpr int PER = NT / 32;
        T v[PER], run = 0;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            v[i] = s_tot[threadIdx.x * PER + i];
            run += v[i];
        }
        T incl = run;
        for (int off = 1; off < 32; off <<= 1) {
            const T u = __shfl_up_sync(0xffffffffu, incl, off);
            if (threadIdx.x >= off) incl += u;
        }
        T ex = incl - run;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const T t = v[i];
            s_tot[threadIdx.x * PER + i] = ex;
            ex += t;
        }
    }
    __syncthreads();
    acc = s_tot[threadIdx.x];
    for (int k = k0; k < min(k0 + seg, L); ++k) {
        R[k] = acc;
        if (k < L - 1) acc += s[base + k];
    }
    __syncthreads();
    for (int i = 0; i < a.nw; ++i) {
        const int w = a.w[i];
        const int64_t tmax = n - w;  // last valid boxcar start
        if (tmax < t0) continue;
        // a threshold beyond T's range can never be met by a window sum that fits T
        const long long thr64 = thr_b[i];
        constexpr long long TMAX = sizeof(T) == 4 ? (long long)INT_MAX : LLONG_MAX;
        constexpr long long TMIN = sizeof(T) == 4 ? (long long)INT_MIN : LLONG_MIN;
        if (thr64 > TMAX) continue;
        const T thr = (T)(thr64 < TMIN ? TMIN : thr64);
        const int64_t tend = min(t0 + TS - 1, tmax);
        for (int64_t t = t0 + threadIdx.x; t <= tend; t += NT) {
            const T B = R[t + w - base] - R[t - base];
            if (B < thr) continue;
            bool ok = true;
            const int64_t lo = max((int64_t)0, t - w + 1), hi = min(tmax, t + w - 1);
            for (int64_t u = lo; u < t && ok; ++u) ok = B > R[u + w - base] - R[u - base];
            for (int64_t u = t + 1; u <= hi && ok; ++u) ok = B >= R[u + w - base] - R[u - base];
            if (!ok) continue;
            const unsigned long long slot = atomicAdd(a.count, 1ull);
            if ((int64_t)slot < a.cap) {
                SpRaw e;
                e.dm_idx = a.dm0 + b;
                e.w = w;
                e.t = t;
                e.B = B;
                a.out[slot] = e;
            }
        }
    }
}

}  // namespace

size_t sp_detect_smem(int wmax, bool narrow) {
    return (size_t)(TS + 3 * wmax) * (narrow ? sizeof(int) : sizeof(long long));
}

// 32-bit prefix sums suffice when the largest sum a tile forms fits
bool sp_narrow(const SpArgs& a) {
    return a.max_value >= 0 && (long long)(TS + 3 * a.wmax) * a.max_value < (1ll << 31) - 1;
}

cudaError_t launch_detect(const SpArgs& a, cudaStream_t s) {
    const bool narrow = sp_narrow(a);
    const size_t shm = sp_detect_smem(a.wmax, narrow);
    const void* k = narrow ? (const void*)k_sp_detect<int> : (const void*)k_sp_detect<long long>;
    cudaError_t e = allow_smem(k, shm);
    if (e != cudaSuccess) return e;
    dim3 gd((unsigned)((a.n + TS - 1) / TS), (unsigned)a.nb);
    if (narrow) k_sp_detect<int><<<gd, NT, shm, s>>>(a);
    else k_sp_detect<long long><<<gd, NT, shm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_single_pulse(const SpArgs& a, unsigned long long* s1, unsigned long long* s2, cudaStream_t s) {
    if (a.nb <= 0 || a.n <= 0) return cudaSuccess;
    if (a.nw < 1 || a.nw > SP_MAXW || a.wmax < 1 || a.wmax > SP_MAXWIDTH) return cudaErrorInvalidValue;
    dim3 gm((unsigned)std::min<int64_t>((a.n + NT - 1) / NT, 64), (unsigned)a.nb);
    k_sp_moments<<<gm, NT, 0, s>>>(a.series, a.stride, a.n, s1, s2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sp_thresholds<<<(unsigned)((a.nb * a.nw + 127) / 128), 128, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_detect(a, s);
}

cudaError_t launch_sp_moments(const int32_t* series, int64_t stride, int64_t n, int32_t nb, unsigned long long* s1,
                              unsigned long long* s2, cudaStream_t s) {
    if (nb <= 0 || n <= 0) return cudaSuccess;
    dim3 gm((unsigned)std::min<int64_t>((n + NT - 1) / NT, 64), (unsigned)nb);
    k_sp_moments<<<gm, NT, 0, s>>>(series, stride, n, s1, s2);
    return cudaGetLastError();
}

cudaError_t launch_sp_detect_only(const SpArgs& a, cudaStream_t s) {
    if (a.nb <= 0 || a.n <= 0) return cudaSuccess;
    return launch_detect(a, s);
}

}  // namespace pss
