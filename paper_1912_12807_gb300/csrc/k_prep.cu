// Filterbank unpack + transpose: file-order samples -> channel-major uint8
// rows of the kept channels, zero-padded to the row pitch.
//
// 8-bit, time-major: sample t of channel c is byte t*nchan + c.
// 1-bit, time-major: channel c of sample t is bit (7 - c%8) of byte
//   t*(nchan/8) + c/8 (most significant bit first), unpacked to 0/1.
// 8-bit, channel-major: rows are copied.
// One HBM pass; 64 x 64 tiles go through shared memory so that both the
// reads (along channels) and the writes (along time) are contiguous.
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
    dim3 grid((unsigned)((a.pitch + TILE - 1) / TILE), (unsigned)((a.ck + TILE - 1) / TILE));
    k_prep<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pss
