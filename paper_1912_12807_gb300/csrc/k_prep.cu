// Filterbank unpack + transpose: file-order samples -> channel-major uint8
// rows of the kept channels, zero-padded to the row pitch.
//
// 8-bit, time-major: sample t of channel c is byte t*nchan + c.
// 1-bit, time-major: channel c of sample t is bit (7 - c%8) of byte
//   t*(nchan/8) + c/8 (most significant bit first), unpacked to 0/1.
// 8-bit, channel-major: rows are copied.
// One HBM pass; 64 x 64 tiles go through shared memory so that both the
// reads (along channels) and the writes (along time) are contiguous.
#include <stdlib.h>

#include "pss_internal.h"

namespace pss {

namespace {

constexpr int TILE = 64;

// one 64 x 64 tile: samples [bx*64, bx*64 + 64) of kept rows [by*64, by*64 + 64)
__device__ __forceinline__ void prep_tile(const PrepArgs& a, int64_t bx, int by) {
    __shared__ uint8_t tile[TILE][TILE + 4];
    const int64_t t0 = bx * TILE;
    const int r0 = by * TILE;
    // read: consecutive threads take consecutive kept channels of one sample
    for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) {
        const int rr = i % TILE, tt = i / TILE;
        const int r = r0 + rr;
        const int64_t t = t0 + tt;
        uint8_t v = 0;
        if (r < a.ck && t < a.nsamp) {
            const int c = a.keep[r];
            if (a.layout == 1) {
                v = a.src[(int64_t)c * a.nsamp + t];
            } else if (a.nbits == 8) {
                v = a.src[t * a.nchan + c];
            } else {
                const uint8_t b = a.src[t * (a.nchan >> 3) + (c >> 3)];
                v = (b >> (7 - (c & 7))) & 1u;
            }
        }
        tile[rr][tt] = v;
    }
    __syncthreads();
    // write: consecutive threads take consecutive samples of one channel
    for (int i = threadIdx.x; i < TILE * TILE; i += blockDim.x) {
        const int tt = i % TILE, rr = i / TILE;
        const int r = r0 + rr;
        const int64_t t = t0 + tt;
        if (r < a.ck && t < a.pitch) a.xcm[(int64_t)r * a.pitch + t] = tile[rr][tt];
    }
}

__global__ void __launch_bounds__(256) k_prep(PrepArgs a) { prep_tile(a, blockIdx.x, blockIdx.y); }

// 8-bit time-major file with every channel kept (row r = channel r): thread
// (group g of 4 channels, run of 16 samples) reads the run's 16 words of its
// 4 channels (a warp: 32 consecutive groups, 128 contiguous bytes per
// sample), transposes each 4 x 4 block of bytes with byte permutes, and
// writes 16 samples of each of its channels as one 16-byte store.  The 8
// warps of a CTA take 8 consecutive runs.
constexpr int U8RUN = 16;

__global__ void __launch_bounds__(256) k_prep_u8(const PrepArgs a) {
    const int ng = a.nchan >> 2;
    const int g = (int)blockIdx.y * 32 + (int)(threadIdx.x & 31);
    const int64_t t0 = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * U8RUN;
    if (g >= ng || t0 >= a.pitch) return;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(a.src);
    uint32_t w[U8RUN];
#pragma unroll
    for (int s = 0; s < U8RUN; ++s) {
        const int64_t t = t0 + s;
        w[s] = t < a.nsamp ? __ldg(src + t * ng + g) : 0u;  // bytes 4g .. 4g + 3 of sample t
    }
    uint32_t o[4][4];  // o[i][q]: channel 4g + i, samples t0 + 4q .. t0 + 4q + 3
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t lo01 = __byte_perm(w[4 * q], w[4 * q + 1], 0x5140);  // s0.c0 s1.c0 s0.c1 s1.c1
        const uint32_t hi01 = __byte_perm(w[4 * q], w[4 * q + 1], 0x7362);  // s0.c2 s1.c2 s0.c3 s1.c3
        const uint32_t lo23 = __byte_perm(w[4 * q + 2], w[4 * q + 3], 0x5140);
        const uint32_t hi23 = __byte_perm(w[4 * q + 2], w[4 * q + 3], 0x7362);
        o[0][q] = __byte_perm(lo01, lo23, 0x5410);  // s0.c0 s1.c0 s2.c0 s3.c0
        o[1][q] = __byte_perm(lo01, lo23, 0x7632);
        o[2][q] = __byte_perm(hi01, hi23, 0x5410);
        o[3][q] = __byte_perm(hi01, hi23, 0x7632);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
        *reinterpret_cast<uint4*>(a.xcm + (int64_t)(4 * g + i) * a.pitch + t0) =
            make_uint4(o[i][0], o[i][1], o[i][2], o[i][3]);
}

// 1-bit time-major file with every channel kept: a warp takes 32
// consecutive samples (one per lane) and walks the channel bytes; for each
// byte, eight ballots give each of its 8 channels' bits over the 32 samples,
// and lane 8 k' + l writes samples 4 l .. 4 l + 3 of channel k = 4 p + k'
// (p = 0, 1) as one 32-bit word of 0/1 bytes: the 4-bit mask times
// 1 + 2^7 + 2^14 + 2^21 puts bit i at bit 8 i (no overlaps), masked to the
// low bit of each byte.
__global__ void __launch_bounds__(256) k_prep_u1(const PrepArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t t0 = ((int64_t)blockIdx.x * 8 + (threadIdx.x >> 5)) * 32;
    if (t0 >= a.pitch) return;  // whole warps
    const int nb = a.nchan >> 3;
    const int64_t t = t0 + lane;
    const int kq = lane >> 3, l = lane & 7;
    for (int cb = 0; cb < nb; ++cb) {
        const uint32_t v = t < a.nsamp ? (uint32_t)a.src[t * nb + cb] : 0u;
        uint32_t mine = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t m = __ballot_sync(0xffffffffu, (v >> (7 - k)) & 1u);
            if (lane == k) mine = m;
        }
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int k = 4 * p + kq;
            const uint32_t m = __shfl_sync(0xffffffffu, mine, k);
            const uint32_t x = (m >> (4 * l)) & 15u;
            *reinterpret_cast<uint32_t*>(a.xcm + (int64_t)(8 * cb + k) * a.pitch + t0 + 4 * l) =
                (x * 0x00204081u) & 0x01010101u;
        }
    }
}

// PSS_PREP_FAST=0 keeps the tiled kernel for every file
bool prep_fast() {
    static const bool on = [] {
        const char* e = getenv("PSS_PREP_FAST");
        return !(e && e[0] == '0');
    }();
    return on;
}

// Work-list form: the files of a group, one launch.  CTA k takes the item
// whose CTA range [first, first + gx * gy) holds k (binary search over the
// items, in order of `first`) and the tile (k - first) of that item's grid.
__global__ void __launch_bounds__(256) k_prep_multi(const PrepItem* items, int nitems) {
    const int64_t k = blockIdx.x;
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].first <= k) lo = mid;
        else hi = mid - 1;
    }
    const PrepItem& it = items[lo];
    const int64_t local = k - it.first;
    const PrepArgs a = it.a;
    prep_tile(a, local % it.gx, (int)(local / it.gx));
}

}  // namespace

int64_t prep_item_ctas(const PrepArgs& a, int32_t* gx) {
    *gx = (int32_t)((a.pitch + TILE - 1) / TILE);
    return (int64_t)*gx * ((a.ck + TILE - 1) / TILE);
}

cudaError_t launch_prep_multi(const PrepItem* items, int nitems, int64_t total_ctas, cudaStream_t s) {
    if (nitems <= 0 || total_ctas <= 0) return cudaSuccess;
    if (total_ctas > 0x7fffffff) return cudaErrorInvalidValue;
    k_prep_multi<<<(unsigned)total_ctas, 256, 0, s>>>(items, nitems);
    return cudaGetLastError();
}

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s) {
    // every channel kept, file order: row r is channel r
    const bool all = a.ck == a.nchan && a.layout == 0 && prep_fast() && (a.pitch & 63) == 0;
    if (all && a.nbits == 8 && (a.nchan & 3) == 0 && ((uintptr_t)a.src & 3) == 0) {
        dim3 g8((unsigned)((a.pitch + 8 * U8RUN - 1) / (8 * U8RUN)), (unsigned)((a.nchan / 4 + 31) / 32));
        k_prep_u8<<<g8, 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    if (all && a.nbits == 1 && (a.nchan & 7) == 0) {
        k_prep_u1<<<(unsigned)((a.pitch + 255) / 256), 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)((a.pitch + TILE - 1) / TILE), (unsigned)((a.ck + TILE - 1) / TILE));
    k_prep<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pss
