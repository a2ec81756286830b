// Harmonic summing, thresholding and candidate compaction (the paper's
// accelsearch, Sect. 2 step 4).
//
// For stage n (1, 2, 4, .., numharm) the plane point (h, j) is taken as the
// n-th harmonic; its k-th harmonic is at half-bin h_k = floor((2kh + n)/(2n))
// and row j_k = Z + sgn(j-Z) floor((2k|j-Z| + n)/(2n)), so
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
    extern __shared__ float S[];  // [(TR+2) * (TH+2)]
    const int SW = TH + 2;
    const int b = blockIdx.z;
    const int64_t h0 = (int64_t)blockIdx.x * TH;
    const int j0 = blockIdx.y * TR;
    const float* P = a.plane + (int64_t)b * a.plane_stride;
    const int halo_n = (TR + 2) * SW;
    const int lane = threadIdx.x & 31;

    for (int si = 0; si < a.nstages; ++si) {
        const int n = 1 << si;
        // update sums on tile + halo
        for (int x = threadIdx.x; x < halo_n; x += NT) {
            const int jr = x / SW, hc = x - jr * SW;
            const int j = j0 - 1 + jr;
            const int64_t h = h0 - 1 + hc;
            if (j < 0 || j >= a.nz || h < 0 || h >= a.nfft) {
                S[x] = -INFINITY;
                continue;
            }
            float acc = (si == 0) ? 0.f : S[x];
            const int d = j - a.Z;
            const int ad = d < 0 ? -d : d;
            const int sg = d < 0 ? -1 : (d > 0 ? 1 : 0);
            for (int k = 1; k <= n; k += (si == 0) ? 1 : 2) {
                const int64_t hk = (2 * (int64_t)k * h + n) / (2 * n);
                const int jk = a.Z + sg * (int)((2 * (int64_t)k * ad + n) / (2 * n));
                acc += __ldg(P + (int64_t)jk * a.nfft + hk);
            }
            S[x] = acc;
        }
        __syncthreads();
        const float thr = a.thr[si];
        const int64_t hmin = a.hmin[si];
        const int npts = TR * TH;
        for (int base = 0; base < npts; base += NT) {
            const int p = base + threadIdx.x;
            bool hit = false;
            int j = 0;
            int64_t h = 0;
            float s = 0.f;
            if (p < npts) {
                const int jr = p / TH, hc = p - jr * TH;
                j = j0 + jr;
                h = h0 + hc;
                if (j < a.nz && h < a.nfft && h >= hmin) {
                    const int x = (jr + 1) * SW + hc + 1;
                    s = S[x];
                    if (s >= thr) {
                        hit = true;
#pragma unroll
                        for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
                            for (int dh = -1; dh <= 1; ++dh) {
                                if (dj == 0 && dh == 0) continue;
                                const float nb = S[x + dj * SW + dh];
                                // neighbour index is larger iff (dj, dh) > (0, 0) lexicographically
                                const bool nb_later = (dj > 0) || (dj == 0 && dh > 0);
                                if (!(s > nb || (s == nb && nb_later))) hit = false;
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
                        c.h = (int32_t)h;
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
    int TR, TH;
    if (a.nz == 1) {
        TR = 1;
        TH = 1024;
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
