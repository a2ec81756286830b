// Folding of candidates' dedispersed series on a grid of trial frequencies
// (the prepfold step, paper Sect. 2 step 6).
//
// One CTA folds one (candidate, trial frequency): sample j has phase
// j x + j^2 g cycles (x = f dt, g = (fdot/2) dt^2) carried in 64-bit fixed
// point (X, G: rint(x 2^64), rint(g 2^64) modulo 2^64, rounded to nearest
// even from the exact binary values of the FP64 x and g formed with
// round-to-nearest intrinsics in the host's order; a negative g wraps),
// phase_j = j X + j^2 G modulo 2^64, and bin floor(phase_j nbin / 2^64) (the
// high word of the 128-bit product): integer arithmetic, so every sample
// lands in the bin the host reading assigns it, with no FP64 per sample.  Each
// thread walks a contiguous run of samples and adds a run of equal bins with
// one shared-memory atomic; the profile and counts are exact integers.
// Thread 0 then forms the reduced chi-square against a flat profile,
// summing the bins in order.
#include "pss_internal.h"

namespace pss {

namespace {

constexpr int NT = 256;

// rint(v 2^64) modulo 2^64, round half to even: v - trunc(v) is exact in FP64
// and lies in (-1, 1), its scaling by 2^64 is exact, and a negative fraction
// wraps (2^64 - rint(|r| 2^64))
__device__ __forceinline__ unsigned long long fixed_point(double v) {
    const double r = __dsub_rn(v, trunc(v));
    if (r >= 0.0) return __double2ull_rn(ldexp(r, 64));
    return 0ull - __double2ull_rn(ldexp(-r, 64));
}

__global__ void __launch_bounds__(NT) k_fold(const __grid_constant__ FoldArgs a) {
    extern __shared__ __align__(16) unsigned long long sm[];  // P [nbin], then n [nbin] (u32)
    unsigned long long* P = sm;
    unsigned int* cnt = reinterpret_cast<unsigned int*>(sm + a.nbin);
    const int r = blockIdx.x / a.nfreq, k = blockIdx.x - r * a.nfreq;
    const FoldItem it = a.items[r];
    for (int b = threadIdx.x; b < a.nbin; b += NT) {
        P[b] = 0ull;
        cnt[b] = 0u;
    }
    __syncthreads();
    const double f = __dadd_rn(it.f, __dmul_rn(__dsub_rn((double)k, __ddiv_rn((double)(a.nfreq - 1), 2.0)),
                                               __ddiv_rn(a.step_bins, it.T)));
    // per-sample phase step x = f dt and drift g = (fdot / 2) dt^2 in 64-bit
    // fixed point (2^-64 cycle, modulo one cycle), rounded to nearest even
    const double x = __dmul_rn(f, it.dt);
    const double g = __dmul_rn(__dmul_rn(0.5, it.fdot), __dmul_rn(it.dt, it.dt));
    const unsigned long long X = fixed_point(x);
    const unsigned long long G = fixed_point(g);
    const unsigned long long nb = (unsigned long long)a.nbin;
    const int32_t* s = a.series + (int64_t)it.row * a.stride;
    const int64_t n = it.n;
    const int64_t per = (n + NT - 1) / NT;
    const int64_t j0 = (int64_t)threadIdx.x * per, j1 = min(n, j0 + per);
    int cur = -1;
    unsigned long long acc = 0ull;
    unsigned int c = 0u;
    for (int64_t j = j0; j < j1; ++j) {
        const unsigned long long ju = (unsigned long long)j;
        const unsigned long long ph = ju * X + (ju * ju) * G;  // wraps modulo 2^64: one cycle
        const int bin = (int)__umul64hi(ph, nb);
        if (bin != cur) {
            if (c) {
                atomicAdd(P + cur, acc);
                atomicAdd(cnt + cur, c);
            }
            cur = bin;
            acc = 0ull;
            c = 0u;
        }
        acc += (unsigned long long)(uint32_t)s[j];
        ++c;
    }
    if (c) {
        atomicAdd(P + cur, acc);
        atomicAdd(cnt + cur, c);
    }
    __syncthreads();
    const int64_t o = (int64_t)blockIdx.x * a.nbin;
    for (int b = threadIdx.x; b < a.nbin; b += NT) {
        a.prof[o + b] = (long long)P[b];
        a.counts[o + b] = (long long)cnt[b];
    }
    if (threadIdx.x == 0) {
        const double fS1 = (double)it.s1, fS2 = (double)it.s2, fN = (double)n;
        const double mu = __ddiv_rn(fS1, fN);
        double var = __ddiv_rn(__dsub_rn(fS2, __ddiv_rn(__dmul_rn(fS1, fS1), fN)), fN);
        double chi = 0.0;
        if (var > 0.0) {
            double sum = 0.0;
            int used = 0;
            for (int b = 0; b < a.nbin; ++b) {
                if (cnt[b] == 0u) continue;
                const double nbv = (double)cnt[b];
                const double d = __dsub_rn((double)(long long)P[b], __dmul_rn(nbv, mu));
                sum = __dadd_rn(sum, __ddiv_rn(__dmul_rn(d, d), __dmul_rn(nbv, var)));
                ++used;
            }
            chi = used > 1 ? __ddiv_rn(sum, (double)(used - 1)) : 0.0;
        }
        a.chi2[blockIdx.x] = chi;
        a.freq[blockIdx.x] = f;
    }
}

}  // namespace

cudaError_t launch_fold(const FoldArgs& a, int64_t nitems, cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    if (a.nbin < 2 || a.nbin > 1024 || a.nfreq < 1 || a.nfreq > 64) return cudaErrorInvalidValue;
    const size_t shm = (size_t)a.nbin * (sizeof(unsigned long long) + sizeof(unsigned int));
    k_fold<<<(unsigned)(nitems * a.nfreq), NT, shm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pss
