// Incoherent dedispersion (paper Sect. 2 step 2: one prepdata run per DM),
// exact in integers:  s[t] = sum_c x[c][t + d_c],  s_ds[j] = sum_{k<ds} s[j*ds+k].
//
// Work decomposition.  A CTA owns G = 16 consecutive DM trials (one warp
// each) and a tile of TN = 1024 native-rate output samples, and walks the
// channels in chunks of CC.  For each channel of a chunk the bytes
// [t0 + min_d, t0 + max_d + TN) that the 16 trials need are fetched once from
// global memory by the bulk-copy (TMA) engine into a shared-memory staging
// area, while the warps are still summing the previous chunk; an mbarrier
// with a byte count signals arrival.  The staged row is then expanded into
// four copies shifted by 0..3 bytes, so every delay is served by aligned
// 32-bit shared-memory reads (consecutive lanes read consecutive words: no
// bank conflicts) and the 16 warps reuse the staged bytes.  Row starts and
// every warp's offsets for all channels are computed once per tile.
//
// Arithmetic is SWAR: a 32-bit word holds 4 consecutive 8-bit samples of one
// channel; (w & 0x00FF00FF) and byte-permute(w) split it into two pairs of
// 16-bit lanes that are added with 32-bit adds.  The adds are issued as
// integer multiply-adds (x * one + acc, `one` a run-time 1) so that they run
// on the FMA pipe while the masks use the integer ALU pipe.  A 16-bit lane
// holds at most 257 * 255 < 65536, so with more than 256 channels the lanes
// are widened into 32-bit accumulators every 256 channels.  The result is the
// exact integer sum.
//
// Every wait on the mbarrier is bounded; on expiry the CTA sets the error
// flag, waits (bounded) for its copies in flight, and exits without writing.
#include "bulk.cuh"
#include "pss_internal.h"

namespace pss {

namespace {

constexpr int G = 16;            // DM trials per CTA (one per warp)
constexpr int KW = 8;            // 32-bit words per lane
constexpr int TN = 32 * 4 * KW;  // native samples per tile (1024)
constexpr int NT = 32 * G;

__device__ __forceinline__ uint32_t madd(uint32_t x, uint32_t one, uint32_t acc) {
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(one), "r"(acc));
    return r;
}

struct Smem {
    uint32_t* copies;  // [CC][4][RW]
    uint8_t* raw;      // [CC][RAWB]
    int32_t* rs;       // [ck] first staged byte of each row, relative to t0 (16-byte aligned absolute)
    uint16_t* offs;    // [G][ck] word index of t0 + d in the row's four shifted copies
    uint64_t* bar;
};

// Shared-memory layout (byte offsets); the same function sizes the launch.
struct Layout {
    size_t copies, raw, rs, offs, bar, total;
};
__host__ __device__ inline Layout layout_of(int RW, int CC, int ck) {
    Layout L;
    const size_t cp = (size_t)CC * 16 * RW, ep = (size_t)G * TN * 4;  // copies / epilogue scratch
    L.copies = 0;
    L.raw = cp > ep ? cp : ep;
    L.rs = L.raw + (size_t)CC * (4 * RW + 16);
    L.offs = L.rs + (size_t)ck * 4;
    L.bar = (L.offs + (size_t)G * ck * 2 + 7) & ~(size_t)7;
    L.total = L.bar + 8;
    return L;
}

// The tile (bx, by, bz) of a launch: time tile bx, trial group by, subband bz.
template <bool INT_OUT, bool WIDE>
__device__ __forceinline__ void dedisp_tile(const DedispArgs& a, int RW, int CC, uint32_t one, int bx, int by,
                                            int bz) {
    extern __shared__ __align__(128) uint8_t smraw[];
    const int RAWB = 4 * RW + 16;
    const Layout Lo = layout_of(RW, CC, a.ck);
    Smem S;
    S.copies = reinterpret_cast<uint32_t*>(smraw + Lo.copies);
    S.raw = smraw + Lo.raw;
    S.rs = reinterpret_cast<int32_t*>(smraw + Lo.rs);
    S.offs = reinterpret_cast<uint16_t*>(smraw + Lo.offs);
    S.bar = reinterpret_cast<uint64_t*>(smraw + Lo.bar);

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int64_t t0 = (int64_t)bx * TN;
    const int g0 = by * G;
    const int gn = min(G, a.nb - g0);
    const int my = g0 + warp;
    const bool active = warp < gn;
    // this CTA's channels: all ck, or subband bz's (stage 1 of the two-stage scheme)
    const uint8_t* xcm = a.xcm;
    const int32_t* delays = a.delays;
    int ck = a.ck;
    int32_t* out_i = a.out_i;
    const int dstride = a.dstride > 0 ? a.dstride : a.ck;
    if (a.zsub) {
        const int2 z = a.zsub[bz];
        xcm += (int64_t)z.x * a.pitch;
        delays += z.x;
        ck = z.y;
        out_i += (int64_t)bz * a.zout;
    }
    const int nchunks = (ck + CC - 1) / CC;

    if (threadIdx.x == 0) {
        mbar_init(S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    // row starts and each warp's offsets for every channel of the tile; an
    // offset past what the staged row holds (a spread larger than the launch
    // was sized for) is refused rather than read out of bounds
    const int omax = 4 * (RW - 32 * KW);
    bool bad = false;
    for (int c = threadIdx.x; c < ck; c += NT) {
        const int32_t* dcol = delays + (int64_t)g0 * dstride + c;
        int32_t dmin = dcol[0];
        for (int g = 1; g < gn; ++g) dmin = min(dmin, dcol[(int64_t)g * dstride]);
        const int64_t st = (t0 + dmin) & ~int64_t(15);
        S.rs[c] = (int32_t)(st - t0);
        // the channel's place in its chunk: its four copies start at word (c mod CC) * 4 RW
        const int base = (c - (c / CC) * CC) * 4 * RW;
        for (int g = 0; g < gn; ++g) {
            const int64_t o = t0 + dcol[(int64_t)g * dstride] - st;
            bad |= (o >= omax);
            // word index into the chunk's copies: copy (o & 3), word (o >> 2) of this channel's
            // (below CC * 4 * RW <= 51200: the copies fill at most 200 KiB)
            S.offs[g * ck + c] = (uint16_t)(bad ? 0 : base + (o & 3) * RW + (o >> 2));
        }
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0 && a.err) atomicExch(a.err, 2);
        return;
    }
    auto issue = [&](int c) {
        // warp 0: one bulk copy per row of the chunk
        if (warp == 0) {
            const int cb = c * CC;
            const int cn = min(CC, ck - cb);
            if (lane == 0) mbar_expect_tx(S.bar, (uint32_t)(cn * RAWB));
            __syncwarp();
            // order this CTA's earlier generic-proxy reads of the staging area
            // before the bulk copies overwrite it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int i = lane; i < cn; i += 32) {
                const uint8_t* src = xcm + (int64_t)(cb + i) * a.pitch + t0 + S.rs[cb + i];
                bulk_g2s(S.raw + (size_t)i * RAWB, src, (uint32_t)RAWB, S.bar);
            }
        }
    };

    uint32_t lo[KW], hi[KW];
    uint32_t wide[WIDE ? 4 * KW : 1];
#pragma unroll
    for (int k = 0; k < KW; ++k) lo[k] = hi[k] = 0u;
#pragma unroll
    for (int k = 0; k < (WIDE ? 4 * KW : 1); ++k) wide[k] = 0u;
    int since_flush = 0;

    __syncthreads();
    issue(0);
    const int qn = RW / 4;
    // expansion work split: qn 16-byte chunks per row, x_rows rows per sweep
    // (rows longer than NT chunks: one row per sweep, chunks strided by NT)
    const int x_rows = qn <= NT ? NT / qn : 1;
    const int x_qstep = qn <= NT ? qn : NT;
    const int x_row = qn <= NT ? (threadIdx.x < x_rows * qn ? (int)threadIdx.x / qn : (1 << 30)) : 0;
    const int x_q = qn <= NT ? (int)threadIdx.x - ((int)threadIdx.x / qn) * qn : (int)threadIdx.x;
    int failed_at = -1;
    for (int c = 0; c < nchunks; ++c) {
        const int cb = c * CC;
        const int cn = min(CC, ck - cb);
        // one warp polls the mbarrier; the others wait at the block barrier (which
        // does not take issue slots), and the barrier passes the staged bytes on
        const bool ok = warp == 0 ? mbar_wait(S.bar, (uint32_t)(c & 1), a.wait_polls) : true;
        if (__syncthreads_or(!ok)) {
            failed_at = c;
            break;
        }
        // expand the staged rows into 4 byte-shifted copies (thread -> (row, 16-byte
        // chunk) split computed once per launch: no division in the loop)
        for (int i = x_row; i < cn; i += x_rows)
        for (int q = x_q; q < qn; q += x_qstep) {
            const uint8_t* src = S.raw + (size_t)i * RAWB + 16 * q;
            const uint4 v = *reinterpret_cast<const uint4*>(src);
            const uint32_t w4 = *reinterpret_cast<const uint32_t*>(src + 16);
            uint32_t* base = S.copies + (size_t)i * 4 * RW + 4 * q;
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
        if (c + 1 < nchunks) issue(c + 1);
        if constexpr (WIDE) {
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
        }
        if (active) {
            const uint16_t* offs = S.offs + warp * ck + cb;
#pragma unroll 4
            for (int i = 0; i < cn; ++i) {
                const uint32_t* p = S.copies + offs[i] + lane;
#pragma unroll
                for (int k = 0; k < KW; ++k) {
                    const uint32_t w = p[32 * k];
                    lo[k] = madd(w & 0x00FF00FFu, one, lo[k]);
                    hi[k] = madd(__byte_perm(w, 0u, 0x4341), one, hi[k]);
                }
            }
        }
        since_flush += cn;
        // no barrier here: the next chunk's first barrier (after its data wait) also orders this
        // chunk's reads of the copies before the next expansion overwrites them
    }
    __syncthreads();  // every warp is done with the copies (the epilogue reuses them)
    if (failed_at >= 0) {
        if (threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
        // let the copies still in flight land before the CTA's shared memory is released
        // (always the full bound, whatever limit the data wait had)
        mbar_wait(S.bar, (uint32_t)(failed_at & 1));
        return;
    }
    uint32_t tot[4 * KW];
#pragma unroll
    for (int k = 0; k < KW; ++k) {
        tot[4 * k + 0] = lo[k] & 0xFFFFu;
        tot[4 * k + 2] = lo[k] >> 16;
        tot[4 * k + 1] = hi[k] & 0xFFFFu;
        tot[4 * k + 3] = hi[k] >> 16;
        if constexpr (WIDE) {
            tot[4 * k + 0] += wide[4 * k + 0];
            tot[4 * k + 2] += wide[4 * k + 2];
            tot[4 * k + 1] += wide[4 * k + 1];
            tot[4 * k + 3] += wide[4 * k + 3];
        }
    }
    if (!active) return;

    // Epilogue.  Lane owns native samples t0 + 4*(lane + 32k) + {0..3}.
    const int64_t j0 = t0 / a.ds;
    unsigned long long part = 0ull;
    if (a.ds == 1) {
        float* of = INT_OUT ? nullptr : a.out_f + (int64_t)my * a.out_stride;
        int32_t* oi = INT_OUT ? out_i + (int64_t)my * a.out_stride : nullptr;
#pragma unroll
        for (int k = 0; k < KW; ++k) {
            const int64_t j = j0 + 4 * (lane + 32 * k);
            if (!INT_OUT && j + 3 < a.nv) {
                part += (unsigned long long)tot[4 * k] + tot[4 * k + 1] + tot[4 * k + 2] + tot[4 * k + 3];
                *reinterpret_cast<float4*>(of + j) =
                    make_float4((float)tot[4 * k], (float)tot[4 * k + 1], (float)tot[4 * k + 2], (float)tot[4 * k + 3]);
                continue;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (j + e < a.nv) {
                    part += tot[4 * k + e];
                    if (INT_OUT) oi[j + e] = (int32_t)tot[4 * k + e];
                    else of[j + e] = (float)tot[4 * k + e];
                }
            }
        }
    } else {
        // boxcar by ds through shared memory: every warp is past the last
        // __syncthreads, so the copy area is free; each warp uses its own slice
        uint32_t* nat = S.copies + (size_t)warp * TN;
#pragma unroll
        for (int k = 0; k < KW; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e) nat[4 * (lane + 32 * k) + e] = tot[4 * k + e];
        __syncwarp();
        const int nout = TN / a.ds;
        for (int oo = lane; oo < nout; oo += 32) {
            const int64_t j = j0 + oo;
            if (j >= a.nv) break;
            unsigned long long acc = 0ull;
            for (int e = 0; e < a.ds; ++e) acc += nat[oo * a.ds + e];
            part += acc;
            if (INT_OUT) out_i[(int64_t)my * a.out_stride + j] = (int32_t)acc;
            else a.out_f[(int64_t)my * a.out_stride + j] = (float)acc;
        }
    }
    if (a.sums) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
        if (lane == 0) atomicAdd(a.sums + my, part);
    }
}

template <bool INT_OUT, bool WIDE>
__global__ void __launch_bounds__(NT) k_dedisp(DedispArgs a, int RW, int CC, uint32_t one) {
    dedisp_tile<INT_OUT, WIDE>(a, RW, CC, one, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Work-list form: every (file, stage, trial run) of a group of files in one
// launch.  CTA k takes the item whose CTA range [first, first + gx * gy)
// holds k (binary search over the items, in order of `first`), and the tile
// (k - first) of that item's grid, with the item's own staging sizes.
template <bool WIDE>
__global__ void __launch_bounds__(NT) k_dedisp_multi(const DedispItem* items, int nitems, uint32_t one) {
    const int64_t k = blockIdx.x;
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].first <= k) lo = mid;
        else hi = mid - 1;
    }
    const DedispItem& it = items[lo];
    const int64_t local = k - it.first;
    const DedispArgs a = it.a;
    dedisp_tile<false, WIDE>(a, it.RW, it.CC, one, (int)(local % it.gx), (int)(local / it.gx), 0);
}

template <bool I, bool W>
cudaError_t launch_t(const DedispArgs& a, dim3 grid, size_t shm, int RW, int CC, cudaStream_t s) {
    cudaError_t e = allow_smem((const void*)k_dedisp<I, W>, shm);
    if (e != cudaSuccess) return e;
    k_dedisp<I, W><<<grid, NT, shm, s>>>(a, RW, CC, 1u);
    return cudaGetLastError();
}

}  // namespace

int dedisp_tile_samples() { return TN; }
int dedisp_group_trials() { return G; }

namespace {
// Launch sizes of a spread: words per staged row copy (RW), channels per
// chunk (CC) and the shared memory; false where the launch is refused.
bool dedisp_sizes(int32_t spread, int32_t ck, int chunk_kb, int* RW_out, int* CC_out, size_t* shm_out) {
    // staged row: the 256 words a lane sweep reads plus the delay spread and
    // the 16-byte alignment slack, in whole 16-byte chunks
    if (spread < 0 || spread > 65535) return false;
    int RW = 32 * KW + (15 + spread) / 4 + 1;
    RW = (RW + 3) & ~3;
    const size_t per_chan = (size_t)16 * RW + (4 * RW + 16);
    const int kb = chunk_kb > 0 ? chunk_kb : 96;  // 96 KiB: two CTAs per SM fit beside the rest
    int CC = (int)(((size_t)kb * 1024) / per_chan);
    if (CC > 32) CC = 32;
    if (CC < 1) CC = 1;
    if (15 + spread > 65535 - 4 * RW) return false;  // offsets are 16-bit
    const size_t shm = layout_of(RW, CC, ck).total;
    if (shm > 220 * 1024) return false;
    *RW_out = RW;
    *CC_out = CC;
    *shm_out = shm;
    return true;
}
}  // namespace

bool dedisp_launch_fits(int32_t spread, int32_t ck, int chunk_kb) {
    int RW, CC;
    size_t shm;
    return dedisp_sizes(spread, ck, chunk_kb, &RW, &CC, &shm);
}

bool dedisp_item(DedispItem* it, int chunk_kb, size_t* shm) {
    const DedispArgs& a = it->a;
    int RW = 0, CC = 0;
    if (a.zsub || a.out_i || !a.out_f) return false;  // the work-list form: exact sums into float rows
    if (!dedisp_sizes(a.spread, a.ck, chunk_kb, &RW, &CC, shm)) return false;
    it->RW = RW;
    it->CC = CC;
    const int64_t L = a.nv * a.ds;
    it->gx = (int32_t)((L + TN - 1) / TN);
    it->gy = (a.nb + G - 1) / G;
    return it->gx > 0 && it->gy > 0;
}

cudaError_t launch_dedisp_multi(const DedispItem* items, int nitems, int64_t total_ctas, size_t shm, bool wide,
                                cudaStream_t s) {
    if (nitems <= 0 || total_ctas <= 0) return cudaSuccess;
    if (total_ctas > 0x7fffffff || shm > 220 * 1024) return cudaErrorInvalidValue;
    const void* fn = wide ? (const void*)k_dedisp_multi<true> : (const void*)k_dedisp_multi<false>;
    cudaError_t e = allow_smem(fn, shm);
    if (e != cudaSuccess) return e;
    if (wide) k_dedisp_multi<true><<<(unsigned)total_ctas, NT, shm, s>>>(items, nitems, 1u);
    else k_dedisp_multi<false><<<(unsigned)total_ctas, NT, shm, s>>>(items, nitems, 1u);
    return cudaGetLastError();
}

cudaError_t launch_dedisp(const DedispArgs& a, int num_sms, cudaStream_t s) {
    (void)num_sms;
    int RW = 0, CC = 0;
    size_t shm = 0;
    if (!dedisp_sizes(a.spread, a.ck, a.chunk_kb, &RW, &CC, &shm)) return cudaErrorInvalidValue;
    const int64_t L = a.nv * a.ds;
    dim3 grid((unsigned)((L + TN - 1) / TN), (unsigned)((a.nb + G - 1) / G), (unsigned)(a.zsub ? a.nz : 1));
    const bool wide = a.ck > 256;
    if (a.out_i) return wide ? launch_t<true, true>(a, grid, shm, RW, CC, s) : launch_t<true, false>(a, grid, shm, RW, CC, s);
    return wide ? launch_t<false, true>(a, grid, shm, RW, CC, s) : launch_t<false, false>(a, grid, shm, RW, CC, s);
}

}  // namespace pss
