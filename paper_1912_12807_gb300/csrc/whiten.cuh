// R2C post-processing of one bin and the exact block lower median with
// whitening by one warp, shared by the whitening kernels and the fused
// spectrum kernel.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_small.cuh"

namespace pss {

constexpr int NBIN = 2048;   // histogram bins on bits 30..20 of the power
constexpr int NCAND = 256;   // candidates gathered from the median's bin

// A_k = (Z_k + conj Z_{M-k}) / 2 - (i/2) e^{-2 pi i k / nfft} (Z_k - conj Z_{M-k}), A_0 = 0
__device__ __forceinline__ float2 r2c_bin(float2 zk, float2 zm, float2 w, int64_t k) {
    const float2 zc = make_float2(zm.x, -zm.y);
    const float2 sum = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
    const float2 dif = make_float2(0.5f * (zk.x - zc.x), 0.5f * (zk.y - zc.y));
    const float2 wd = cmul(w, dif);
    float2 a = make_float2(sum.x + wd.y, sum.y - wd.x);  // sum - i * w * dif
    if (k == 0) a = make_float2(0.f, 0.f);
    return a;
}

// One warp whitens one block of W = 32 VPL bins held in registers (lane l
// holds bins k0 + l + 32 i): the lower median (rank (m-1)/2) of |A|^2 is
// selected exactly from a private histogram of the float bit patterns
// (bits 30..20), the candidates of the median's bin gathered and ranked
// (ties by position), with radix rounds on the remaining bits if that bin
// is crowded; the block is scaled by sqrt(ln 2 / med) (or 1 if !whiten),
// written to Oblk[lane + 32 i], and ln 2 / med stored in *gain_out
// (nullable).  The bin with k0 + l + 32 i == 0 (DC) is excluded.
template <int VPL>
__device__ __forceinline__ void whiten_block(float2 (&A)[VPL], int64_t k0, int lane, int m, uint32_t* hist,
                                             uint32_t* cand, uint32_t* cpos, int whiten, float* gain_out,
                                             float2* Oblk) {
    auto keyof = [&](int i) -> uint32_t {
        return (k0 == 0 && lane == 0 && i == 0) ? 0xFFFFFFFFu : __float_as_uint(pow2(A[i]));
    };
    __syncwarp();
    for (int i = lane; i < NBIN; i += 32) hist[i] = 0u;
    __syncwarp();
#pragma unroll
    for (int i = 0; i < VPL; ++i) {
        const uint32_t kk = keyof(i);
        if (kk != 0xFFFFFFFFu) atomicAdd(&hist[kk >> 20], 1u);
    }
    __syncwarp();
    const uint32_t rank0 = (uint32_t)((m - 1) / 2);
    // the bin holding rank0: lane l owns bins [l * NBIN/32, (l+1) * NBIN/32)
    constexpr int BPL = NBIN / 32;
    uint32_t tot = 0;
#pragma unroll 8
    for (int i = 0; i < BPL; ++i) tot += hist[lane * BPL + ((i + lane) & (BPL - 1))];  // rotated: no bank conflicts
    uint32_t incl = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    const uint32_t before0 = incl - tot;
    const bool mine = rank0 >= before0 && rank0 < incl;
    const int owner = __ffs(__ballot_sync(0xffffffffu, mine)) - 1;
    uint32_t bin = 0, rank = 0;
    if (lane == owner) {
        uint32_t before = before0;
        for (int i = 0; i < BPL; ++i) {
            const uint32_t c = hist[lane * BPL + i];
            if (rank0 < before + c) {
                bin = (uint32_t)(lane * BPL + i);
                rank = rank0 - before;
                break;
            }
            before += c;
        }
    }
    bin = __shfl_sync(0xffffffffu, bin, owner);
    rank = __shfl_sync(0xffffffffu, rank, owner);
    const uint32_t nin = hist[bin];
    uint32_t med_bits = 0;
    if (nin <= (uint32_t)NCAND) {
        // gather the bin's values with their positions, then count ranks (ties by position)
        uint32_t base = 0;
#pragma unroll
        for (int i = 0; i < VPL; ++i) {
            const uint32_t kk = keyof(i);
            const bool in = kk != 0xFFFFFFFFu && (kk >> 20) == bin;
            const unsigned bal = __ballot_sync(0xffffffffu, in);
            if (in) {
                const uint32_t slot = base + __popc(bal & ((1u << lane) - 1u));
                cand[slot] = kk;
                cpos[slot] = (uint32_t)(lane + 32 * i);
            }
            base += __popc(bal);
        }
        __syncwarp();
        uint32_t found = 0;
        bool have = false;
        for (uint32_t c = lane; c < nin; c += 32) {
            const uint32_t v = cand[c], pv = cpos[c];
            uint32_t r = 0;
            for (uint32_t q = 0; q < nin; ++q) {
                const uint32_t u = cand[q];
                r += (u < v) || (u == v && cpos[q] < pv);
            }
            if (r == rank) {
                found = v;
                have = true;
            }
        }
        const int who = __ffs(__ballot_sync(0xffffffffu, have)) - 1;
        med_bits = __shfl_sync(0xffffffffu, found, who < 0 ? 0 : who);
    } else {
        // many values share the top bits: radix rounds on bits 19..0 (8, 8, 4)
        uint32_t prefix = bin << 20, mask = 0xFFF00000u, rk = rank;
#pragma unroll
        for (int pass = 0; pass < 3; ++pass) {
            const int shift = pass == 0 ? 12 : (pass == 1 ? 4 : 0);
            const uint32_t dmask = pass == 2 ? 15u : 255u;
            __syncwarp();
            for (int i = lane; i < 256; i += 32) hist[i] = 0u;
            __syncwarp();
#pragma unroll
            for (int i = 0; i < VPL; ++i) {
                const uint32_t kk = keyof(i);
                if (kk != 0xFFFFFFFFu && (kk & mask) == prefix) atomicAdd(&hist[(kk >> shift) & dmask], 1u);
            }
            __syncwarp();
            uint32_t dsel = 0, rsel = 0;
            if (lane == 0) {
                uint32_t before = 0;
                for (uint32_t d = 0; d <= dmask; ++d) {
                    if (rk < before + hist[d]) {
                        dsel = d;
                        rsel = rk - before;
                        break;
                    }
                    before += hist[d];
                }
            }
            dsel = __shfl_sync(0xffffffffu, dsel, 0);
            rsel = __shfl_sync(0xffffffffu, rsel, 0);
            prefix |= dsel << shift;
            mask |= dmask << shift;
            rk = rsel;
        }
        med_bits = prefix;
    }
    // scale sqrt(ln 2 / med) and gain ln 2 / med in FP64, once per warp (FP64 is slow)
    float scale = 1.f;
    if (lane == 0) {
        const float med = __uint_as_float(med_bits);
        const double g = med > 0.f ? 0.69314718055994530942 / (double)med : 0.0;
        scale = whiten ? (float)sqrt(g) : 1.f;
        if (gain_out) *gain_out = (float)g;
    }
    scale = __shfl_sync(0xffffffffu, scale, 0);
#pragma unroll
    for (int i = 0; i < VPL; ++i) Oblk[lane + 32 * i] = make_float2(A[i].x * scale, A[i].y * scale);
}

// The same block whitening by a pair of warps (h = 0, 1) that share one
// histogram: lane l of warp h holds bins k0 + h*32*VPL + l + 32 i.  The
// selected element, the scale and the output are those of whiten_block on
// the same 2*32*VPL bins (positions h*32*VPL + l + 32 i order ties the same
// way).  The pair synchronises with named barrier `bar` (64 threads).
// sh: NBIN + 2*NCAND + 8 words of shared memory for the pair.  With Oblk
// null the scaled bins stay in A.  Returns the scale.
__device__ __forceinline__ void pair_sync(int bar) { asm volatile("bar.sync %0, 64;" ::"r"(bar) : "memory"); }

template <int VPL>
__device__ __forceinline__ float whiten_block_pair(float2 (&A)[VPL], int64_t k0, int h, int lane, int m, uint32_t* sh,
                                                   int bar, int whiten, float* gain_out, float2* Oblk) {
    uint32_t* hist = sh;
    uint32_t* cand = sh + NBIN;
    uint32_t* cpos = cand + NCAND;
    uint32_t* misc = cpos + NCAND;  // [0] warp-0 total, [1] bin, [2] rank, [3] slots, [4] value, [5] scale bits
    const int t = h * 32 + lane;     // 0..63
    auto keyof = [&](int i) -> uint32_t {
        return (k0 == 0 && t == 0 && i == 0) ? 0xFFFFFFFFu : __float_as_uint(pow2(A[i]));
    };
    for (int i = t; i < NBIN; i += 64) hist[i] = 0u;
    if (t == 0) misc[3] = 0u;
    pair_sync(bar);
#pragma unroll
    for (int i = 0; i < VPL; ++i) {
        const uint32_t kk = keyof(i);
        if (kk != 0xFFFFFFFFu) atomicAdd(&hist[kk >> 20], 1u);
    }
    pair_sync(bar);
    const uint32_t rank0 = (uint32_t)((m - 1) / 2);
    // thread t owns bins [t * BPT, (t+1) * BPT)
    constexpr int BPT = NBIN / 64;
    uint32_t tot = 0;
#pragma unroll 8
    for (int i = 0; i < BPT; ++i) tot += hist[t * BPT + ((i + t) & (BPT - 1))];  // rotated: no bank conflicts
    uint32_t incl = tot;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (h == 0 && lane == 31) misc[0] = incl;
    pair_sync(bar);
    if (h == 1) incl += misc[0];
    const uint32_t before0 = incl - tot;
    if (rank0 >= before0 && rank0 < incl) {
        uint32_t before = before0;
        for (int i = 0; i < BPT; ++i) {
            const uint32_t c = hist[t * BPT + i];
            if (rank0 < before + c) {
                misc[1] = (uint32_t)(t * BPT + i);
                misc[2] = rank0 - before;
                break;
            }
            before += c;
        }
    }
    pair_sync(bar);
    const uint32_t bin = misc[1], rank = misc[2];
    const uint32_t nin = hist[bin];
    if (nin <= (uint32_t)NCAND) {
#pragma unroll
        for (int i = 0; i < VPL; ++i) {
            const uint32_t kk = keyof(i);
            if (kk != 0xFFFFFFFFu && (kk >> 20) == bin) {
                const uint32_t slot = atomicAdd(&misc[3], 1u);
                cand[slot] = kk;
                cpos[slot] = (uint32_t)(h * 32 * VPL + lane + 32 * i);
            }
        }
        pair_sync(bar);
        for (uint32_t c = t; c < nin; c += 64) {
            const uint32_t v = cand[c], pv = cpos[c];
            uint32_t r = 0;
            for (uint32_t q = 0; q < nin; ++q) {
                const uint32_t u = cand[q];
                r += (u < v) || (u == v && cpos[q] < pv);
            }
            if (r == rank) misc[4] = v;
        }
    } else {
        // many values share the top bits: radix rounds on bits 19..0 (8, 8, 4)
        uint32_t prefix = bin << 20, mask = 0xFFF00000u, rk = rank;
#pragma unroll
        for (int pass = 0; pass < 3; ++pass) {
            const int shift = pass == 0 ? 12 : (pass == 1 ? 4 : 0);
            const uint32_t dmask = pass == 2 ? 15u : 255u;
            pair_sync(bar);
            for (int i = t; i < 256; i += 64) hist[i] = 0u;
            pair_sync(bar);
#pragma unroll
            for (int i = 0; i < VPL; ++i) {
                const uint32_t kk = keyof(i);
                if (kk != 0xFFFFFFFFu && (kk & mask) == prefix) atomicAdd(&hist[(kk >> shift) & dmask], 1u);
            }
            pair_sync(bar);
            if (t == 0) {
                uint32_t before = 0;
                for (uint32_t d = 0; d <= dmask; ++d) {
                    if (rk < before + hist[d]) {
                        misc[1] = d;
                        misc[2] = rk - before;
                        break;
                    }
                    before += hist[d];
                }
            }
            pair_sync(bar);
            prefix |= misc[1] << shift;
            mask |= dmask << shift;
            rk = misc[2];
        }
        if (t == 0) misc[4] = prefix;
    }
    pair_sync(bar);
    // scale sqrt(ln 2 / med) and gain ln 2 / med in FP64, once per pair (FP64 is slow)
    if (t == 0) {
        const float med = __uint_as_float(misc[4]);
        const double g = med > 0.f ? 0.69314718055994530942 / (double)med : 0.0;
        misc[5] = __float_as_uint(whiten ? (float)sqrt(g) : 1.f);
        if (gain_out) *gain_out = (float)g;
    }
    pair_sync(bar);
    const float scale = __uint_as_float(misc[5]);
    if (Oblk) {
#pragma unroll
        for (int i = 0; i < VPL; ++i) Oblk[h * 32 * VPL + lane + 32 * i] = make_float2(A[i].x * scale, A[i].y * scale);
    } else {
#pragma unroll
        for (int i = 0; i < VPL; ++i) A[i] = make_float2(A[i].x * scale, A[i].y * scale);
    }
    return scale;
}

}  // namespace pss
