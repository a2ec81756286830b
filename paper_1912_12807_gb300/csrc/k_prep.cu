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

__global__ void __launch_bounds__(256) k_prep(PrepArgs a) {
    __shared__ uint8_t tile[TILE][TILE + 4];
    const int64_t t0 = (int64_t)blockIdx.x * TILE;
    const int r0 = blockIdx.y * TILE;
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

}  // namespace

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s) {
    dim3 grid((unsigned)((a.pitch + TILE - 1) / TILE), (unsigned)((a.ck + TILE - 1) / TILE));
    k_prep<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pss
