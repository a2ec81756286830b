// Two-stage (subband) dedispersion, stage 2 (the prepsubband scheme, paper
// Sect. 5):  s_i[t] = sum_b u_{g(i),b}[t + D_b(i)],  then the ds boxcar.
// Stage 1 (the per-subband sums u at each group's nominal DM) is the
// dedispersion kernel run with one subband per blockIdx.z (k_dedisp.cu).
//
// A CTA owns one group row of stage-1 sums and a tile of TN native samples;
// its 16 warps are 16 trials of the group (more trials: further passes).
// For every subband the samples [t0 + Dmin_b, t0 + TN + Dmax_b) of the
// group's row, which all of the group's trials read, are staged once in
// shared memory by one bulk (TMA engine) copy per row, from the 16-byte
// boundary at or below t0 + Dmin_b, completed on an mbarrier whose wait is
// bounded (on expiry the CTA sets the error flag and leaves); then each warp
// adds the row at its own offset D_b(i) - Dmin_b (lane l: samples l + 32 j,
// consecutive words across lanes).  The sums are exact int32.  Copies may
// read up to RW samples past a row's end: the stage-1 buffer carries that
// much slack after its last row.
#include "bulk.cuh"
#include "pss_internal.h"

namespace pss {

namespace {

constexpr int TN = 1024;        // native samples per tile
constexpr int NW = 16;          // warps (trials) per pass
constexpr int NT = 32 * NW;
constexpr int KJ = TN / 32;     // samples per lane
constexpr int MAXSB = 64;       // subbands staged per round

template <bool INT_OUT>
__global__ void __launch_bounds__(NT, 2) k_subsum(const __grid_constant__ SubsumArgs a, int RW, int SBC) {
    extern __shared__ __align__(128) int32_t sm[];  // [SBC][RW] staged rows; reused by the ds epilogue
    __shared__ int32_t s_dmin[MAXSB], s_lead[MAXSB];
    __shared__ __align__(8) uint64_t s_bar;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.y;
    const int2 gr = a.grp[r];
    const int first = gr.x - a.b0rel;  // the group's first trial relative to the batch
    const int tlo = max(0, first), thi = min(a.nb, first + gr.y);
    const int64_t t0 = (int64_t)blockIdx.x * TN;
    const int32_t* urow = a.u + (int64_t)r * a.u_rowstride;
    const int64_t j0 = t0 / a.ds;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t phase = 0;
    for (int p0 = tlo; p0 < thi; p0 += NW) {
        const int pn = min(NW, thi - p0);
        const int my = p0 + warp;
        const bool active = warp < pn;
        int32_t acc[KJ];
#pragma unroll
        for (int j = 0; j < KJ; ++j) acc[j] = 0;
        for (int sb0 = 0; sb0 < a.nsub; sb0 += SBC) {
            const int sbn = min(SBC, a.nsub - sb0);
            if (threadIdx.x < sbn) {
                int32_t dmin = a.D[(int64_t)p0 * a.nsub + sb0 + threadIdx.x];
                for (int k = 1; k < pn; ++k) dmin = min(dmin, a.D[(int64_t)(p0 + k) * a.nsub + sb0 + threadIdx.x]);
                s_dmin[threadIdx.x] = dmin;
                // rows are staged from a 16-byte boundary: `lead` samples before t0 + dmin
                s_lead[threadIdx.x] = (int32_t)((t0 + dmin) & 3);
            }
            __syncthreads();
            // one bulk copy per subband row of RW samples (the group's window plus alignment slack)
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&s_bar, (uint32_t)(sbn * RW * 4));
                for (int b = 0; b < sbn; ++b) {
                    const int64_t st = t0 + s_dmin[b] - s_lead[b];
                    bulk_g2s(sm + (size_t)b * RW, urow + (int64_t)(sb0 + b) * a.u_zstride + st, (uint32_t)(RW * 4),
                             &s_bar);
                }
            }
            const bool ok = warp == 0 ? mbar_wait(&s_bar, phase, a.wait_polls) : true;
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
                mbar_wait(&s_bar, phase ^ 1u);  // let the copies in flight land before leaving (full bound)
                return;
            }
            if (active) {
                const int32_t* drow = a.D + (int64_t)my * a.nsub + sb0;
                for (int b = 0; b < sbn; ++b) {
                    const int32_t* row = sm + (size_t)b * RW + (drow[b] - s_dmin[b] + s_lead[b]) + lane;
#pragma unroll
                    for (int j = 0; j < KJ; ++j) acc[j] += row[32 * j];
                }
            }
            __syncthreads();
        }
        unsigned long long part = 0ull;
        if (a.ds == 1) {
            if (active) {
#pragma unroll
                for (int j = 0; j < KJ; ++j) {
                    const int64_t t = j0 + lane + 32 * j;
                    if (t < a.nv) {
                        part += (unsigned long long)(uint32_t)acc[j];
                        if (INT_OUT) a.out_i[(int64_t)my * a.out_stride + t] = acc[j];
                        else a.out_f[(int64_t)my * a.out_stride + t] = (float)acc[j];
                    }
                }
            }
        } else {
            // boxcar by ds through shared memory (each warp its own TN slice)
            int32_t* nat = sm + (size_t)warp * TN;
            if (active) {
#pragma unroll
                for (int j = 0; j < KJ; ++j) nat[lane + 32 * j] = acc[j];
            }
            __syncwarp();
            if (active) {
                const int nout = TN / a.ds;
                for (int oo = lane; oo < nout; oo += 32) {
                    const int64_t j = j0 + oo;
                    if (j >= a.nv) break;
                    unsigned long long v = 0ull;
                    for (int e = 0; e < a.ds; ++e) v += (uint32_t)nat[oo * a.ds + e];
                    part += v;
                    if (INT_OUT) a.out_i[(int64_t)my * a.out_stride + j] = (int32_t)v;
                    else a.out_f[(int64_t)my * a.out_stride + j] = (float)v;
                }
            }
            __syncthreads();  // the slices are staging space again in the next pass
        }
        if (a.sums && active) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            if (lane == 0) atomicAdd(a.sums + my, part);
        }
    }
}

}  // namespace

cudaError_t launch_subsum(const SubsumArgs& a, cudaStream_t s) {
    if (a.nb <= 0 || a.ngrp <= 0) return cudaSuccess;
    if (a.spread < 0 || a.ds < 1 || a.ds > TN || (TN % a.ds) != 0) return cudaErrorInvalidValue;
    // window TN + spread, plus up to 3 samples of alignment lead, in whole 16-byte units
    const int RW = (TN + a.spread + 3 + 3) & ~3;
    // subbands per staging round: about 96 KiB of rows, at least one
    int SBC = (int)((96 * 1024) / ((size_t)RW * 4));
    SBC = std::max(1, std::min(std::min(SBC, MAXSB), a.nsub));
    const size_t shm = std::max((size_t)SBC * RW, (size_t)NW * TN) * sizeof(int32_t);
    if (shm > 220 * 1024) return cudaErrorInvalidValue;
    const int64_t L = a.nv * a.ds;
    dim3 grid((unsigned)((L + TN - 1) / TN), (unsigned)a.ngrp);
    if (a.out_i) {
        cudaError_t e = allow_smem((const void*)k_subsum<true>, shm);
        if (e != cudaSuccess) return e;
        k_subsum<true><<<grid, NT, shm, s>>>(a, RW, SBC);
    } else {
        cudaError_t e = allow_smem((const void*)k_subsum<false>, shm);
        if (e != cudaSuccess) return e;
        k_subsum<false><<<grid, NT, shm, s>>>(a, RW, SBC);
    }
    return cudaGetLastError();
}

}  // namespace pss
