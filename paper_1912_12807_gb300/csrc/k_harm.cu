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
#include <stdlib.h>

#include "pss_internal.h"

namespace pss {

namespace {

constexpr int NT = 256;

struct Tile {
    int h0, j0, jlo, r0, halo_n, nfft, lane, b;
    const float* P;
};

// Stage SI (n = 2^SI): add the odd harmonics to the sums held in S, then
// test and compact the tile's points.  TR x TH is the tile; ONE_ROW is the
// zmax = 0 case (a single plane row, no row arithmetic).
template <int SI, int TR, int TH, bool ONE_ROW>
__device__ __forceinline__ void harm_stage(const HarmArgs& a, const Tile& t, float* S, const float* s_thr,
                                           const int* s_hmin) {
    constexpr int n = 1 << SI;
    constexpr int sh = SI + 1;
    constexpr int SW = TH + 2;
    for (int x = threadIdx.x; x < t.halo_n; x += NT) {
        const int rr = ONE_ROW ? 0 : x / SW;
        const int hc = ONE_ROW ? x : x - rr * SW;
        const int j = t.jlo + rr;
        const int h = t.h0 - 1 + hc;
        float* dst = S + (t.r0 + rr) * SW + hc;
        if (h < 0 || h >= t.nfft) {
            *dst = -INFINITY;
            continue;
        }
        float acc;
        if constexpr (SI == 0) {
            acc = __ldg(t.P + (ONE_ROW ? 0 : j * t.nfft) + h);
        } else {
            // the n/2 odd harmonics: independent loads, issued together
            float v[n / 2];
            const int h2 = 2 * h;
            if constexpr (ONE_ROW) {
#pragma unroll
                for (int q = 0; q < n / 2; ++q) v[q] = __ldg(t.P + (((2 * q + 1) * h2 + n) >> sh));
            } else {
                const int d = j - a.Z;
                const int ad2 = 2 * (d < 0 ? -d : d);
#pragma unroll
                for (int q = 0; q < n / 2; ++q) {
                    const int k = 2 * q + 1;
                    const int dk = (k * ad2 + n) >> sh;
                    const int jk = d < 0 ? a.Z - dk : a.Z + dk;
                    v[q] = __ldg(t.P + jk * t.nfft + ((k * h2 + n) >> sh));
                }
            }
            acc = *dst;
#pragma unroll
            for (int q = 0; q < n / 2; ++q) acc += v[q];
        }
        *dst = acc;
    }
    __syncthreads();
    const float thr = s_thr[SI];
    const int hmin = s_hmin[SI];
    constexpr int npts = TR * TH;
#pragma unroll 1
    for (int base = 0; base < npts; base += NT) {
        const int p = base + threadIdx.x;
        bool hit = false;
        int j = 0, h = 0;
        float s = 0.f;
        if (p < npts) {
            const int jr = p / TH, hc = p - jr * TH;
            j = t.j0 + jr;
            h = t.h0 + hc;
            if (j < a.nz && h < t.nfft && h >= hmin) {
                const int x = (jr + 1) * SW + hc + 1;
                s = S[x];
                if (s >= thr) {
                    hit = true;
#pragma unroll
                    for (int dj = -1; dj <= 1; ++dj) {
                        if (ONE_ROW && dj != 0) continue;
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
            if (t.lane == 0) slot0 = atomicAdd(a.counter, (unsigned long long)__popc(m));
            slot0 = __shfl_sync(0xffffffffu, slot0, 0);
            if (hit) {
                const unsigned long long slot = slot0 + __popc(m & ((1u << t.lane) - 1u));
                if ((int64_t)slot < a.cap) {
                    pss_raw_cand c;
                    c.dm_idx = a.row_dm ? a.row_dm[t.b] : a.dm0 + t.b;
                    c.numharm = n;
                    c.h = h;
                    c.j = j;
                    c.power = s;
                    c.reserved = a.row_file ? a.row_file[t.b] : 0;
                    a.out[slot] = c;
                }
            }
        }
    }
    __syncthreads();
}

template <int SI, int NSTAGES, int TR, int TH, bool ONE_ROW>
__device__ __forceinline__ void harm_stages(const HarmArgs& a, const Tile& t, float* S, const float* s_thr,
                                            const int* s_hmin) {
    if constexpr (SI < NSTAGES) {
        harm_stage<SI, TR, TH, ONE_ROW>(a, t, S, s_thr, s_hmin);
        harm_stages<SI + 1, NSTAGES, TR, TH, ONE_ROW>(a, t, S, s_thr, s_hmin);
    }
}

template <int NSTAGES, int TR, int TH, bool ONE_ROW>
__global__ void __launch_bounds__(NT) k_harm(const __grid_constant__ HarmArgs a) {
    __shared__ float S[(TR + 2) * (TH + 2)];  // row r <-> j = j0 - 1 + r
    __shared__ float s_thr[8];
    __shared__ int s_hmin[8];
#pragma unroll
    for (int q = 0; q < 6; ++q)
        if (threadIdx.x == q) {  // constant indices keep the parameter block out of local memory
            s_thr[q] = a.thr[q];
            s_hmin[q] = a.row_hmin ? a.row_hmin[8 * blockIdx.z + q] : a.hmin[q];
        }
    Tile t;
    t.b = blockIdx.z;
    t.h0 = blockIdx.x * TH;
    t.j0 = blockIdx.y * TR;
    t.nfft = (int)a.nfft;
    t.P = a.plane + (int64_t)t.b * a.plane_stride;
    // rows of the plane present in tile + halo
    t.jlo = ONE_ROW ? 0 : max(t.j0 - 1, 0);
    const int jhi = ONE_ROW ? 1 : min(t.j0 + TR + 1, a.nz);
    t.r0 = t.jlo - (t.j0 - 1);
    t.halo_n = (jhi - t.jlo) * (TH + 2);
    t.lane = threadIdx.x & 31;
    __syncthreads();
    harm_stages<0, NSTAGES, TR, TH, ONE_ROW>(a, t, S, s_thr, s_hmin);
}

template <int TR, int TH, bool ONE_ROW>
cudaError_t launch_variant(const HarmArgs& a, cudaStream_t s) {
    dim3 grid((unsigned)((a.nfft + TH - 1) / TH), (unsigned)((a.nz + TR - 1) / TR), (unsigned)a.nb);
    switch (a.nstages) {
        case 1: k_harm<1, TR, TH, ONE_ROW><<<grid, NT, 0, s>>>(a); break;
        case 2: k_harm<2, TR, TH, ONE_ROW><<<grid, NT, 0, s>>>(a); break;
        case 3: k_harm<3, TR, TH, ONE_ROW><<<grid, NT, 0, s>>>(a); break;
        case 4: k_harm<4, TR, TH, ONE_ROW><<<grid, NT, 0, s>>>(a); break;
        case 5: k_harm<5, TR, TH, ONE_ROW><<<grid, NT, 0, s>>>(a); break;
        case 6: k_harm<6, TR, TH, ONE_ROW><<<grid, NT, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---- register-blocked variant ------------------------------------------------
//
// A warp owns WR = 32 R consecutive half-bins of one plane row j; lane l
// holds the sums of the points h = hw + l + 32 i (i < R) in registers.  For
// stage n and odd harmonic k, point (h, j) reads row j_k (the same for the
// whole warp) at half-bin (2kh + n) >> (s+1); stepping h by 32 steps that
// index by exactly 32k/n (an integer for n <= 32), so one index computation
// per harmonic serves all R points and the loads use compile-time offsets,
// each coalesced across the warp.  Additions happen in the order of k_harm
// (stage by stage, odd k increasing), so the sums are bit-identical.
// Threshold tests run on the lane's maximum; a warp with a point above
// threshold takes same-row neighbours from adjacent lanes and recomputes any
// other neighbour (warp edges, rows j +- 1) from the plane.

// S_n at (h, j) from the plane (the same additions in the same order).
template <int SI>
__device__ float harm_sum_at(const float* P, int h, int j, int nfft, int nz, int Z) {
    if (h < 0 || h >= nfft || j < 0 || j >= nz) return -INFINITY;
    float acc = __ldg(P + j * nfft + h);
    const int d = j - Z, ad2 = 2 * (d < 0 ? -d : d);
#pragma unroll
    for (int s = 1; s <= SI; ++s) {
        const int n = 1 << s;
        for (int q = 0; q < n / 2; ++q) {
            const int k = 2 * q + 1;
            const int dk = (k * ad2 + n) >> (s + 1);
            const int jk = d < 0 ? Z - dk : Z + dk;
            acc += __ldg(P + jk * nfft + ((2 * k * h + n) >> (s + 1)));
        }
    }
    return acc;
}

template <int SI, int R>
__device__ __forceinline__ void reg_test(const HarmArgs& a, const float* P, const float (&acc)[R], int hw, int j,
                                         int lane, int b) {
    const float thr = a.thr[SI];
    float mx = acc[0];
#pragma unroll
    for (int i = 1; i < R; ++i) mx = fmaxf(mx, acc[i]);
    if (!__any_sync(0xffffffffu, mx >= thr)) return;
    const int nfft = (int)a.nfft, hmin = a.row_hmin ? a.row_hmin[8 * b + SI] : a.hmin[SI], nz = a.nz, Z = a.Z;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        float left = __shfl_up_sync(0xffffffffu, acc[i], 1);
        float right = __shfl_down_sync(0xffffffffu, acc[i], 1);
        const float l31 = __shfl_sync(0xffffffffu, acc[i > 0 ? i - 1 : 0], 31);
        const float r0 = __shfl_sync(0xffffffffu, acc[i < R - 1 ? i + 1 : R - 1], 0);
        const float s = acc[i];
        const int h = hw + lane + 32 * i;
        if (s >= thr && h >= hmin) {
            if (lane == 0) left = i > 0 ? l31 : harm_sum_at<SI>(P, hw - 1, j, nfft, nz, Z);
            if (lane == 31) right = i < R - 1 ? r0 : harm_sum_at<SI>(P, hw + 32 * R, j, nfft, nz, Z);
            // strictly above every earlier neighbour, ties to the lower index against later ones
            bool hit = s > left && s >= right;
            if (nz > 1) {
#pragma unroll
                for (int dh = -1; dh <= 1; ++dh) {
                    if (!hit) break;
                    hit = s > harm_sum_at<SI>(P, h + dh, j - 1, nfft, nz, Z) &&
                          s >= harm_sum_at<SI>(P, h + dh, j + 1, nfft, nz, Z);
                }
            }
            if (hit) {
                const unsigned long long slot = atomicAdd(a.counter, 1ull);
                if ((int64_t)slot < a.cap) {
                    pss_raw_cand c;
                    c.dm_idx = a.row_dm ? a.row_dm[b] : a.dm0 + b;
                    c.numharm = 1 << SI;
                    c.h = h;
                    c.j = j;
                    c.power = s;
                    c.reserved = a.row_file ? a.row_file[b] : 0;
                    a.out[slot] = c;
                }
            }
        }
    }
}

template <int SI, int NSTAGES, int R>
__device__ __forceinline__ void reg_stages(const HarmArgs& a, const float* P, float (&acc)[R], int hw, int j,
                                           int lane, int b) {
    if constexpr (SI < NSTAGES) {
        if constexpr (SI > 0) {
            constexpr int n = 1 << SI;
            const int d = j - a.Z, ad2 = 2 * (d < 0 ? -d : d);
#pragma unroll
            for (int q = 0; q < n / 2; ++q) {
                const int k = 2 * q + 1;
                const int dk = (k * ad2 + n) >> (SI + 1);
                const int jk = d < 0 ? a.Z - dk : a.Z + dk;
                const float* p = P + jk * (int)a.nfft + ((2 * k * (hw + lane) + n) >> (SI + 1));
#pragma unroll
                for (int i = 0; i < R; ++i) acc[i] += __ldg(p + (32 / n) * k * i);
            }
        }
        reg_test<SI, R>(a, P, acc, hw, j, lane, b);
        reg_stages<SI + 1, NSTAGES, R>(a, P, acc, hw, j, lane, b);
    }
}

constexpr int REG_NT = 128;

template <int NSTAGES, int R, bool ROWS>
__global__ void __launch_bounds__(REG_NT) k_harm_reg(const __grid_constant__ HarmArgs a) {
    // blocks of consecutive launch order take the same h range of successive
    // rows, so the harmonic rows they read overlap while they are in L2; with
    // ROWS the warps of a block take consecutive rows of one h range, so the
    // harmonic rows they share are read through the same L1
    const int lane = threadIdx.x & 31;
    const int j = ROWS ? blockIdx.x * (REG_NT / 32) + (threadIdx.x >> 5) : blockIdx.x;
    if (ROWS && j >= a.nz) return;  // no barriers in this kernel
    const int b = blockIdx.z;
    const int hw = ROWS ? blockIdx.y * 32 * R : (blockIdx.y * (REG_NT / 32) + (threadIdx.x >> 5)) * 32 * R;
    const float* P = a.plane + (int64_t)b * a.plane_stride;
    float acc[R];
    const float* row = P + j * (int)a.nfft;
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = __ldg(row + hw + lane + 32 * i);
    reg_stages<0, NSTAGES, R>(a, P, acc, hw, j, lane, b);
}

// 2-D planes: the warps of a block take consecutive plane rows (default; 31.1 -> 28.9 ms on
// the zmax 200 accel file); PSS_HARM_ROWS=0 keeps one row per block
bool harm_rows() {
    static const int v = [] {
        const char* e = getenv("PSS_HARM_ROWS");
        return e ? (e[0] == '1' ? 1 : 0) : 1;
    }();
    return v == 1;
}

template <int R, bool ROWS>
cudaError_t launch_reg_t(const HarmArgs& a, cudaStream_t s) {
    constexpr int W = REG_NT / 32;
    dim3 grid(ROWS ? (unsigned)((a.nz + W - 1) / W) : (unsigned)a.nz,
              ROWS ? (unsigned)(a.nfft / (32 * R)) : (unsigned)(a.nfft / (REG_NT * R)), (unsigned)a.nb);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    switch (a.nstages) {
        case 1: k_harm_reg<1, R, ROWS><<<grid, REG_NT, 0, s>>>(a); break;
        case 2: k_harm_reg<2, R, ROWS><<<grid, REG_NT, 0, s>>>(a); break;
        case 3: k_harm_reg<3, R, ROWS><<<grid, REG_NT, 0, s>>>(a); break;
        case 4: k_harm_reg<4, R, ROWS><<<grid, REG_NT, 0, s>>>(a); break;
        case 5: k_harm_reg<5, R, ROWS><<<grid, REG_NT, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int R>
cudaError_t launch_reg(const HarmArgs& a, cudaStream_t s) {
    if (a.nz > 1 && harm_rows() && a.nfft / (32 * R) <= 65535) return launch_reg_t<R, true>(a, s);
    return launch_reg_t<R, false>(a, s);
}

}  // namespace

cudaError_t launch_harm(const HarmArgs& a, cudaStream_t s) {
    if (a.nfft > (int64_t(1) << 24) || a.nstages > 6) return cudaErrorInvalidValue;
    if ((int64_t)a.nz * a.nfft > (int64_t(1) << 31)) return cudaErrorInvalidValue;  // 32-bit plane offsets
    // register-blocked kernel: up to 16 harmonics, whole warps of 32 x 16 points
    if (a.run == 8 && a.nstages <= 5 && a.nfft % (REG_NT * 8) == 0 && a.nfft / (REG_NT * 8) <= 65535 &&
        a.nb <= 65535)
        return launch_reg<8>(a, s);
    if (a.nstages <= 5 && a.nfft % (REG_NT * 16) == 0 && a.nfft / (REG_NT * 16) <= 65535 && a.nb <= 65535)
        return launch_reg<16>(a, s);
    if (a.nz == 1) return launch_variant<1, 2048, true>(a, s);
    return launch_variant<4, 256, false>(a, s);
}

}  // namespace pss
