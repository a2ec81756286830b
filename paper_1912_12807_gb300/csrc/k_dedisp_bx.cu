// Dedispersion of downsampled plan rows through a per-channel boxcar table
// (paper Sect. 2 step 2 with the downsampling of Tables 2-3), exact in
// integers.  With W_c[t] = sum_{k<ds} x[c][t + k] the downsampled series is
//
//     s_ds[j] = sum_c sum_{k<ds} x[c][j ds + d_c + k] = sum_c W_c[j ds + d_c],
//
// one term per channel and output sample instead of ds.  The table is laid
// out by phase, Wt[c][p][m] = W_c[m ds + p], so that with d_c = q ds + p a
// trial reads, for channel c, the contiguous run Wt[c][p][q + j], j < N_v:
// consecutive lanes read consecutive 16-bit words.  W_c[t] <= 255 ds fits 16
// bits for ds <= 256; the channel sum is accumulated in 32 bits.
//
// k_bx_table: one CTA per (channel, run of MT table columns) stages the
// MT ds + ds input bytes it needs, forms their prefix sums in shared
// memory (stored with a skew of one word per ds so that the strided reads of
// one phase row hit distinct banks) and writes W as differences of two
// prefix sums, row by row (coalesced).
//
// k_dedisp_bx: a CTA owns GW consecutive trials (one warp each) and a tile
// of TJ output samples; the lanes of a warp turn 32 channels' delays into
// table offsets at once (ds is a power of two: a shift and a mask each) and
// pass them round by shuffle.
// Adjacent trials mostly share a channel's phase row and offset, so their
// warps read the same lines through L1.
#include "pss_internal.h"

namespace pss {

namespace {

constexpr int TB_NT = 256;     // table builder threads
constexpr int TB_SPAN = 8192;  // native samples per table-builder CTA, plus a tail of ds
constexpr int GW = 8;          // trials (warps) per dedispersion CTA
constexpr int KJ = 8;          // outputs per lane
constexpr int TJ = 32 * KJ;    // outputs per tile

__device__ __forceinline__ int skew(int k, int lds) { return k + (k >> lds); }

// ds = 2^lds <= 256 (plan rows are powers of two), MT = 2^lmt columns, so a
// CTA covers MT ds = TB_SPAN bytes of its channel plus a tail of ds bytes.
__global__ void __launch_bounds__(TB_NT) k_bx_table(const __grid_constant__ BxTableArgs a) {
    extern __shared__ __align__(16) unsigned char tb_sm[];
    const int lds = a.lds, ds = 1 << lds, lmt = a.lmt, MT = 1 << lmt;
    const int span = MT << lds;  // TB_SPAN
    const int L = span + ds;     // columns [m0, m0 + MT) need x[t0 .. t0 + L)
    uint8_t* xb = tb_sm;                                               // [L] staged bytes
    int32_t* P = reinterpret_cast<int32_t*>(tb_sm + ((L + 15) & ~15));  // skewed prefix sums P[0..L]
    __shared__ int32_t s_warp[TB_NT / 32];
    const int c = blockIdx.y;
    const int64_t m0 = (int64_t)blockIdx.x * MT;
    const int64_t t0 = m0 << lds;
    const uint8_t* row = a.xcm + (int64_t)c * a.pitch;
    if (t0 + L <= a.nsamp) {
        // row starts and t0 are 16-byte aligned (pitch is a multiple of 64, t0 of TB_SPAN)
        const uint4* src = reinterpret_cast<const uint4*>(row + t0);
        for (int k = threadIdx.x; k < span / 16; k += TB_NT) reinterpret_cast<uint4*>(xb)[k] = __ldg(src + k);
        for (int k = span + threadIdx.x; k < L; k += TB_NT) xb[k] = row[t0 + k];
    } else {
        for (int k = threadIdx.x; k < L; k += TB_NT) xb[k] = (t0 + k < a.nsamp) ? row[t0 + k] : (uint8_t)0;
    }
    __syncthreads();
    // exclusive prefix sums of the first `span` bytes: 32 per thread, then a block scan
    constexpr int SEG = TB_SPAN / TB_NT;
    const int k0 = threadIdx.x * SEG;
    int32_t v[SEG];
    int32_t tot = 0;
#pragma unroll
    for (int q = 0; q < SEG / 16; ++q) {
        const uint4 w = reinterpret_cast<const uint4*>(xb + k0)[q];
        const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            v[16 * q + e] = (int32_t)((ww[e >> 2] >> (8 * (e & 3))) & 0xFFu);
            tot += v[16 * q + e];
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t incl = tot;
    for (int off = 1; off < 32; off <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += u;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int32_t run = incl - tot;
    for (int w = 0; w < warp; ++w) run += s_warp[w];
#pragma unroll
    for (int e = 0; e < SEG; ++e) {
        P[skew(k0 + e, lds)] = run;
        run += v[e];
    }
    if (warp == 0) {
        // the tail P[span .. L]: a warp scan of the last ds bytes (at most 8 per lane)
        int32_t base = 0;
        for (int w = 0; w < TB_NT / 32; ++w) base += s_warp[w];
        const int per = (ds + 31) >> 5;
        int32_t loc[BX_MAX_DS / 32];
        int32_t t = 0;
#pragma unroll
        for (int e = 0; e < BX_MAX_DS / 32; ++e) {
            const int i = lane * per + e;
            loc[e] = (e < per && i < ds) ? (int32_t)xb[span + i] : 0;
            t += loc[e];
        }
        int32_t in = t;
        for (int off = 1; off < 32; off <<= 1) {
            const int32_t u = __shfl_up_sync(0xffffffffu, in, off);
            if (lane >= off) in += u;
        }
        int32_t r = base + in - t;
#pragma unroll
        for (int e = 0; e < BX_MAX_DS / 32; ++e) {
            const int i = lane * per + e;
            if (e < per && i < ds) P[skew(span + i, lds)] = r;
            r += loc[e];
        }
        if (lane == 31) P[skew(L, lds)] = base + in;
    }
    __syncthreads();
    // W_c[m ds + p] = P[(m - m0) ds + p + ds] - P[(m - m0) ds + p], written by phase rows
    uint16_t* out = a.table + (int64_t)c * ds * a.mstride;
    const int64_t ncol = min((int64_t)MT, a.mlen - m0);
    for (int idx = threadIdx.x; idx < span; idx += TB_NT) {
        const int p = idx >> lmt, mm = idx & (MT - 1);
        if (mm >= ncol) continue;
        const int k = (mm << lds) + p;
        out[(int64_t)p * a.mstride + m0 + mm] = (uint16_t)(P[skew(k + ds, lds)] - P[skew(k, lds)]);
    }
}

template <bool INT_OUT>
__global__ void __launch_bounds__(32 * GW) k_dedisp_bx(const __grid_constant__ BxArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int my = blockIdx.y * GW + warp;
    if (my >= a.nb) return;
    const int64_t j0 = (int64_t)blockIdx.x * TJ;
    const int32_t* dl = a.delays + (int64_t)my * a.ck;
    const uint16_t* __restrict__ tab = a.table;
    const bool full = j0 + TJ <= a.nv;
    uint32_t acc[KJ];
#pragma unroll
    for (int k = 0; k < KJ; ++k) acc[k] = 0u;
    for (int cb = 0; cb < a.ck; cb += 32) {
        // lane l: the table offset of channel cb + l for this trial at output j0
        int64_t o = 0;
        if (cb + lane < a.ck) {
            const int32_t d = __ldg(dl + cb + lane);
            const int32_t q = d >> a.lds, p = d & ((1 << a.lds) - 1);
            o = (((int64_t)(cb + lane) << a.lds) + p) * a.mstride + q + j0;
        }
        const int cn = min(32, a.ck - cb);
        if (full) {
            for (int i = 0; i < cn; ++i) {
                const uint16_t* src = tab + __shfl_sync(0xffffffffu, o, i) + lane;
#pragma unroll
                for (int k = 0; k < KJ; ++k) acc[k] += __ldg(src + 32 * k);
            }
        } else {
            for (int i = 0; i < cn; ++i) {
                const uint16_t* src = tab + __shfl_sync(0xffffffffu, o, i) + lane;
#pragma unroll
                for (int k = 0; k < KJ; ++k)
                    if (j0 + lane + 32 * k < a.nv) acc[k] += __ldg(src + 32 * k);
            }
        }
    }
    unsigned long long part = 0ull;
#pragma unroll
    for (int k = 0; k < KJ; ++k) {
        const int64_t j = j0 + lane + 32 * k;
        if (j < a.nv) {
            part += acc[k];
            if (INT_OUT) a.out_i[(int64_t)my * a.out_stride + j] = (int32_t)acc[k];
            else a.out_f[(int64_t)my * a.out_stride + j] = (float)acc[k];
        }
    }
    if (a.sums) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if (lane == 0) atomicAdd(a.sums + my, part);
    }
}

}  // namespace

int bx_table_cols(int ds) { return TB_SPAN / std::max(ds, 1); }

cudaError_t launch_bx_table(const BxTableArgs& a, cudaStream_t s) {
    if (a.ck <= 0 || a.mlen <= 0) return cudaSuccess;
    const int ds = 1 << a.lds;
    // grid.y is the channel: at most 65535 rows
    if (a.lds < 1 || ds > BX_MAX_DS || (1 << a.lmt) != bx_table_cols(ds) || a.mstride < a.mlen || (a.pitch & 15) ||
        a.ck > 65535)
        return cudaErrorInvalidValue;
    const int L = TB_SPAN + ds;
    const size_t shm = (size_t)((L + 15) & ~15) + (size_t)(L + 1 + (L >> a.lds) + 2) * sizeof(int32_t);
    cudaError_t e = allow_smem((const void*)k_bx_table, shm);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((a.mlen + (1 << a.lmt) - 1) >> a.lmt), (unsigned)a.ck);
    k_bx_table<<<grid, TB_NT, shm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dedisp_bx(const BxArgs& a, cudaStream_t s) {
    if (a.nb <= 0 || a.nv <= 0) return cudaSuccess;
    if (a.lds < 1 || (1 << a.lds) > BX_MAX_DS || a.ck <= 0) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((a.nv + TJ - 1) / TJ), (unsigned)((a.nb + GW - 1) / GW));
    if (a.out_i) k_dedisp_bx<true><<<grid, 32 * GW, 0, s>>>(a);
    else k_dedisp_bx<false><<<grid, 32 * GW, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pss
