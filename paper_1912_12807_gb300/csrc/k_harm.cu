// Harmonic summing, thresholding and candidate compaction (the paper's
// accelsearch, Sect. 2 step 4).
//
// For stage n = 2^s (1, 2, 4, .., numharm) the plane point (h, j) is taken
// as the n-th harmonic; its k-th harmonic is at half-bin
// h_k = floor((2kh + n)/(2n)) = (2kh + n) >> (s+1) and row
// j_k = Z + sgn(j-Z) ((2k|j-Z| + n) >> (s+1)), so
//   S_n(h, j) = sum_{k=1..n} P[j_k][h_k].
// Because h_{2m} at stage n equals h_m at stage n/2 (and likewise for rows),
// S_n = S_{n/2} + sum over odd k of P[j_k][h_k]: each stage adds only its odd
// harmonics to the previous stage's sums, kept in shared memory.
//
// A CTA owns a tile of TR rows x TH half-bins and keeps S for the tile plus
// a one-point halo, so the 3x3 local-maximum test (strictly larger than
// every in-plane neighbour, exact ties to the lower linear index j*nfft+h)
// needs no second pass.  Points that pass the stage threshold and the
// f >= f_lo cut are compacted with a warp ballot and one atomic per warp;
// the global counter always counts, so an overflow of `cap` is detected.
#include <math.h>

#include "pss_internal.h"

namespace pss {

namespace {

constexpr int NT = 256;

__global__ void __launch_bounds__(NT) k_harm(HarmArgs a, int TR, int TH) {
    extern __shared__ float S[];  // [(TR+2) * (TH+2)], row r <-> j = j0 - 1 + r
    __shared__ float s_thr[8];
    __shared__ int s_hmin[8];
    if (threadIdx.x < 8) {
        const int i = threadIdx.x < a.nstages ? threadIdx.x : 0;
        s_thr[threadIdx.x] = a.thr[i];
        s_hmin[threadIdx.x] = a.hmin[i];
    }
    const int SW = TH + 2;
    const int b = blockIdx.z;
    const int h0 = blockIdx.x * TH;
    const int j0 = blockIdx.y * TR;
    const int nfft = (int)a.nfft;
    const float* P = a.plane + (int64_t)b * a.plane_stride;
    // rows of the plane present in tile + halo
    const int jlo = max(j0 - 1, 0), jhi = min(j0 + TR + 1, a.nz);
    const int r0 = jlo - (j0 - 1);
    const int nrows = jhi - jlo;
    const int halo_n = nrows * SW;
    const int lane = threadIdx.x & 31;

    for (int si = 0; si < a.nstages; ++si) {
        const int n = 1 << si;
        const int sh = si + 1;
        for (int x = threadIdx.x; x < halo_n; x += NT) {
            const int rr = x / SW, hc = x - rr * SW;
            const int j = jlo + rr;
            const int h = h0 - 1 + hc;
            float* dst = S + (r0 + rr) * SW + hc;
            if (h < 0 || h >= nfft) {
                *dst = -INFINITY;
                continue;
            }
            const int d = j - a.Z;
            const int ad = d < 0 ? -d : d;
            float acc;
            if (si == 0) {
                acc = __ldg(P + (int64_t)j * nfft + h);
            } else {
                acc = *dst;
                for (int k = 1; k < n; k += 2) {
                    const int hk = (2 * k * h + n) >> sh;
                    const int dk = (2 * k * ad + n) >> sh;
                    const int jk = d < 0 ? a.Z - dk : a.Z + dk;
                    acc += __ldg(P + (int64_t)jk * nfft + hk);
                }
            }
            *dst = acc;
        }
        __syncthreads();
        const float thr = s_thr[si];
        const int hmin = s_hmin[si];
        const int npts = TR * TH;
        for (int base = 0; base < npts; base += NT) {
            const int p = base + threadIdx.x;
            bool hit = false;
            int j = 0, h = 0;
            float s = 0.f;
            if (p < npts) {
                const int jr = p / TH, hc = p - jr * TH;
                j = j0 + jr;
                h = h0 + hc;
                if (j < a.nz && h < nfft && h >= hmin) {
                    const int x = (jr + 1) * SW + hc + 1;
                    s = S[x];
                    if (s >= thr) {
                        hit = true;
#pragma unroll
                        for (int dj = -1; dj <= 1; ++dj) {
                            if (j + dj < 0 || j + dj >= a.nz) continue;
#pragma unroll
                            for (int dh = -1; dh <= 1; ++dh) {
                                if (dj == 0 && dh == 0) continue;
                                const float nb = S[x + dj * SW + dh];
                                // the neighbour's linear index is larger iff (dj, dh) > (0, 0)
                                const bool nb_later = (dj > 0) || (dj == 0 && dh > 0);
                                if (!(s > nb || (s == nb && nb_later))) hit = false;
                            }
                        }
                    }
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (m) {
                unsigned long long slot0 = 0ull;
                if (lane == 0) slot0 = atomicAdd(a.counter, (unsigned long long)__popc(m));
                slot0 = __shfl_sync(0xffffffffu, slot0, 0);
                if (hit) {
                    const unsigned long long slot = slot0 + __popc(m & ((1u << lane) - 1u));
                    if ((int64_t)slot < a.cap) {
                        pss_raw_cand c;
                        c.dm_idx = a.dm0 + b;
                        c.numharm = n;
                        c.h = h;
                        c.j = j;
                        c.power = s;
                        c.reserved = 0;
                        a.out[slot] = c;
                    }
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_harm(const HarmArgs& a, cudaStream_t s) {
    if (a.nfft > (int64_t(1) << 24) || a.nstages > 6) return cudaErrorInvalidValue;
    int TR, TH;
    if (a.nz == 1) {
        TR = 1;
        TH = 2048;
    } else {
        TR = 4;
        TH = 256;
    }
    const size_t shm = (size_t)(TR + 2) * (TH + 2) * sizeof(float);
    dim3 grid((unsigned)((a.nfft + TH - 1) / TH), (unsigned)((a.nz + TR - 1) / TR), (unsigned)a.nb);
    k_harm<<<grid, NT, shm, s>>>(a, TR, TH);
    return cudaGetLastError();
}

}  // namespace pss
