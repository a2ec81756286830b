// Incoherent dedispersion (paper Sect. 2 step 2: one prepdata run per DM),
// exact in integers:  s[t] = sum_c x[c][t + d_c],  s_ds[j] = sum_{k<ds} s[j*ds+k].
//
// Work decomposition.  A CTA owns G = 8 consecutive DM trials (one warp
// each) and a tile of TN = 1024 native-rate output samples.  Channels are
// processed in chunks of CC: for every channel of the chunk the bytes
// [t0 + min_d, t0 + max_d + TN) that the 8 trials need are staged once in
// shared memory and reused by all 8 warps.  Each row is stored as four
// copies shifted by 0..3 bytes, so any delay is served by aligned 32-bit
// shared-memory reads (consecutive lanes read consecutive words: no bank
// conflicts).
//
// Arithmetic is SWAR: a 32-bit word holds 4 consecutive 8-bit samples of one
// channel; (w & 0x00FF00FF) and (w >> 8) & 0x00FF00FF split it into two
// pairs of 16-bit lanes that are added with ordinary 32-bit adds.  A 16-bit
// lane holds at most 257 * 255 < 65536, so the lanes are widened into 32-bit
// accumulators every 256 channels.  The result is the exact integer sum.
#include "pss_internal.h"

namespace pss {

namespace {

constexpr int G = 8;            // DM trials per CTA (one per warp)
constexpr int KW = 8;           // 32-bit words per lane
constexpr int TN = 32 * 4 * KW; // native samples per tile (1024)

__device__ __forceinline__ uint32_t hi_pairs(uint32_t w) {
    // bytes 1 and 3 of w into the low bytes of two 16-bit lanes
    return __byte_perm(w, 0u, 0x4341);
}

template <bool INT_OUT>
__global__ void __launch_bounds__(256) k_dedisp(DedispArgs a, int RW, int CC) {
    extern __shared__ __align__(16) uint32_t smem[];
    // smem layout: [CC][4 copies][RW words] staged rows, then per-channel a16
    int64_t* row_start = reinterpret_cast<int64_t*>(smem + (size_t)CC * 4 * RW);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * TN;
    const int g0 = blockIdx.y * G;
    const int gn = min(G, a.nb - g0);
    const int my = g0 + warp;  // this warp's trial in the batch
    const bool active = warp < gn;
    const int32_t* drow = a.delays + (int64_t)(active ? my : g0) * a.ck;

    uint32_t lo[KW], hi[KW];
    uint32_t wide[4 * KW];
#pragma unroll
    for (int k = 0; k < KW; ++k) lo[k] = hi[k] = 0u;
#pragma unroll
    for (int k = 0; k < 4 * KW; ++k) wide[k] = 0u;
    int since_flush = 0;

    const int qn = RW / 4;  // 16-byte chunks per copy row
    for (int cb = 0; cb < a.ck; cb += CC) {
        const int cn = min(CC, a.ck - cb);
        // per-channel first staged byte (16-byte aligned)
        for (int i = threadIdx.x; i < cn; i += blockDim.x) {
            const int32_t* dcol = a.delays + (int64_t)g0 * a.ck + cb + i;
            int32_t dmin = dcol[0];
            for (int g = 1; g < gn; ++g) dmin = min(dmin, dcol[(int64_t)g * a.ck]);
            row_start[i] = (t0 + dmin) & ~int64_t(15);
        }
        __syncthreads();
        // stage: 4 byte-shifted copies of each row
        for (int it = threadIdx.x; it < cn * qn; it += blockDim.x) {
            const int i = it / qn, q = it - i * qn;
            const uint8_t* src = a.xcm + (int64_t)(cb + i) * a.pitch + row_start[i] + 16 * q;
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(src));
            const uint32_t w4 = __ldg(reinterpret_cast<const uint32_t*>(src + 16));
            uint32_t* base = smem + (size_t)i * 4 * RW + 4 * q;
            const uint32_t W[5] = {v.x, v.y, v.z, v.w, w4};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                uint4 o;
                o.x = __funnelshift_r(W[0], W[1], 8 * s);
                o.y = __funnelshift_r(W[1], W[2], 8 * s);
                o.z = __funnelshift_r(W[2], W[3], 8 * s);
                o.w = __funnelshift_r(W[3], W[4], 8 * s);
                *reinterpret_cast<uint4*>(base + (size_t)s * RW) = o;
            }
        }
        __syncthreads();
        if (since_flush + cn > 256) {
#pragma unroll
            for (int k = 0; k < KW; ++k) {
                wide[4 * k + 0] += lo[k] & 0xFFFFu;
                wide[4 * k + 2] += lo[k] >> 16;
                wide[4 * k + 1] += hi[k] & 0xFFFFu;
                wide[4 * k + 3] += hi[k] >> 16;
                lo[k] = hi[k] = 0u;
            }
            since_flush = 0;
        }
        if (active) {
            for (int i = 0; i < cn; ++i) {
                const int64_t o = t0 + drow[cb + i] - row_start[i];
                const uint32_t* p = smem + ((size_t)i * 4 + (o & 3)) * RW + (o >> 2) + lane;
#pragma unroll
                for (int k = 0; k < KW; ++k) {
                    const uint32_t w = p[32 * k];
                    lo[k] += w & 0x00FF00FFu;
                    hi[k] += hi_pairs(w);
                }
            }
        }
        since_flush += cn;
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        wide[4 * k + 0] += lo[k] & 0xFFFFu;
        wide[4 * k + 2] += lo[k] >> 16;
        wide[4 * k + 1] += hi[k] & 0xFFFFu;
        wide[4 * k + 3] += hi[k] >> 16;
    }
    if (!active) return;

    // Epilogue.  Lane owns native samples t0 + 4*(lane + 32k) + {0..3}.
    const int64_t j0 = t0 / a.ds;  // first output of this tile
    unsigned long long part = 0ull;
    if (a.ds == 1) {
        float* of = INT_OUT ? nullptr : a.out_f + (int64_t)my * a.out_stride;
        int32_t* oi = INT_OUT ? a.out_i + (int64_t)my * a.out_stride : nullptr;
#pragma unroll
        for (int k = 0; k < KW; ++k) {
            const int64_t j = j0 + 4 * (lane + 32 * k);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (j + e < a.nv) {
                    part += wide[4 * k + e];
                    if (INT_OUT) oi[j + e] = (int32_t)wide[4 * k + e];
                    else of[j + e] = (float)wide[4 * k + e];
                }
            }
        }
    } else {
        // boxcar by ds through shared memory (the staging area is free now;
        // each warp uses its own TN-word slice, so a warp barrier suffices)
        uint32_t* nat = smem + (size_t)warp * TN;
#pragma unroll
        for (int k = 0; k < KW; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e) nat[4 * (lane + 32 * k) + e] = wide[4 * k + e];
        __syncwarp();
        const int nout = TN / a.ds;
        for (int oo = lane; oo < nout; oo += 32) {
            const int64_t j = j0 + oo;
            if (j >= a.nv) break;
            unsigned long long acc = 0ull;
            for (int e = 0; e < a.ds; ++e) acc += nat[oo * a.ds + e];
            part += acc;
            if (INT_OUT) a.out_i[(int64_t)my * a.out_stride + j] = (int32_t)acc;
            else a.out_f[(int64_t)my * a.out_stride + j] = (float)acc;
        }
    }
    if (a.sums) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if (lane == 0) atomicAdd(a.sums + my, part);
    }
}

}  // namespace

int dedisp_tile_samples() { return TN; }

cudaError_t launch_dedisp(const DedispArgs& a, int num_sms, cudaStream_t s) {
    (void)num_sms;
    // staged row: 256 words read per lane sweep plus the delay spread and
    // the 16-byte alignment slack, in whole 16-byte chunks
    int RW = 32 * KW + (15 + a.spread) / 4 + 1;
    RW = (RW + 3) & ~3;
    const size_t per_chan = (size_t)4 * RW * 4;
    int CC = (int)((96 * 1024) / per_chan);
    if (CC > 32) CC = 32;
    if (CC < 1) CC = 1;
    size_t shm = (size_t)CC * per_chan + (size_t)CC * sizeof(int64_t);
    if (shm < (size_t)G * TN * 4 + CC * sizeof(int64_t)) shm = (size_t)G * TN * 4 + CC * sizeof(int64_t);
    if (shm > 200 * 1024) return cudaErrorInvalidValue;
    const int64_t L = a.nv * a.ds;
    dim3 grid((unsigned)((L + TN - 1) / TN), (unsigned)((a.nb + G - 1) / G));
    if (a.out_i) {
        cudaFuncSetAttribute(k_dedisp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        k_dedisp<true><<<grid, 256, shm, s>>>(a, RW, CC);
    } else {
        cudaFuncSetAttribute(k_dedisp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        k_dedisp<false><<<grid, 256, shm, s>>>(a, RW, CC);
    }
    return cudaGetLastError();
}

}  // namespace pss
