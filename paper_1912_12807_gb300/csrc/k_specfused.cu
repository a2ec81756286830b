// Fused spectrum of one DM trial on a 16-CTA thread-block cluster: mean
// subtraction, the M = 2^17 point complex FFT of the packed real series
// (nfft = 2^18), R2C post-processing, block-median whitening and the zmax = 0
// half-bin plane, with the spectrum kept in the cluster's distributed shared
// memory instead of making five passes over HBM (paper Sect. 2 steps 3-4;
// the arithmetic is that of k_fft_pass, k_r2c_whiten and k_plane_z0).
//
// Four-step FFT with M = 16 x 8192: for n = 8192 n1 + n2 and k = k1 + 16 k2,
//   X[k1 + 16 k2] = sum_{n2} W_8192^{n2 k2} (W_M^{n2 k1} sum_{n1} z[8192 n1 + n2] W_16^{n1 k1}).
// CTA r of the cluster:
//   A. loads columns n2 = 512 r + j (j < 512, one per thread), does the
//      16-point DFTs over n1, applies W_M^{n2 k1} and stores element
//      (k1, n2) into CTA k1's shared buffer B at n2;
//   B. transforms its row k1 = r in place (8192 points, radix 8-8-8-8-2);
//   C. gathers the contiguous bins k = 8192 r + u from the rows of all 16
//      CTAs into its buffer A;
//   D. forms A_k from X_k and the mirror X_{M-k} (read from CTA 15 - r),
//      then whitens its 8 blocks of 1024 bins, one warp each;
//   E. builds a tile of its whitened bins with 15 / 16 bins of halo from
//      the neighbouring CTAs and writes both half-bins of every bin.
// Cluster barriers separate the phases; a CTA reads and writes other CTAs'
// shared memory only between barriers that all 16 have reached.
#include <cooperative_groups.h>

#include "fft_small.cuh"
#include "pss_internal.h"
#include "whiten.cuh"

namespace cg = cooperative_groups;

namespace pss {

namespace {

constexpr int CL = 16;          // CTAs per cluster (N1)
constexpr int N2 = 8192;        // points per CTA
constexpr int MF = CL * N2;     // complex points per trial (nfft / 2)
constexpr int FT = 512;         // threads per CTA
constexpr int NTAP = 32;        // z = 0 half-bin FIR taps (m = 16)
constexpr int RUN = N2 / FT;    // bins per thread in the FIR (16)
constexpr int TILE = N2 + NTAP - 1;
constexpr int TILE_PAD = TILE + TILE / 16 + 1;  // one spare slot per 16 (odd stride per thread)
constexpr int NW = 8;           // whitening warps (one 1024-bin block each)

// shared-memory layout (float2 units unless noted)
constexpr size_t OFF_A = 0;                       // [TILE_PAD]  contiguous slice / FIR tile
constexpr size_t OFF_B = OFF_A + TILE_PAD;        // [N2]        row of the FFT / whitened slice
constexpr size_t OFF_WH = OFF_B + N2;             // [128]
constexpr size_t OFF_WL = OFF_WH + 128;           // [64]
constexpr size_t OFF_U32 = OFF_WL + 64;           // uint32 area: hist [NW][NBIN], cand, cpos [NW][NCAND]
constexpr size_t SMEM_BYTES = OFF_U32 * sizeof(float2) + (size_t)NW * (NBIN + 2 * NCAND) * sizeof(uint32_t);

__device__ __forceinline__ int tp(int i) { return i + (i >> 4); }  // padded FIR tile index

// exp(-2 pi i t / 8192) = WH[t >> 6] WL[t & 63]
__device__ __forceinline__ float2 tw8192(const float2* WH, const float2* WL, int t) {
    return cmul(WH[t >> 6], WL[t & 63]);
}

// One in-place Stockham sub-stage (radix RR, running span NS) of the
// 8192-point FFT held in shared memory with the fp() swizzle.
template <int RR, int NS>
__device__ __forceinline__ void substage8192(float2* buf, const float2* WH, const float2* WL) {
    constexpr int NB = N2 / RR;
    constexpr int PER = NB / FT;
    float2 x[PER][RR];
    int dst[PER];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * FT;
        const int k = b & (NS - 1);
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            x[p][q] = buf[fp(b + q * NB)];
            if (NS > 1 && q && k) x[p][q] = cmul(x[p][q], tw8192(WH, WL, q * k * (N2 / (RR * NS))));
        }
        dst[p] = (b - k) * RR + k;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        dft_small<RR>(x[p]);
#pragma unroll
        for (int q = 0; q < RR; ++q) buf[fp(dst[p] + q * NS)] = x[p][q];
    }
    __syncthreads();
}

__global__ void __launch_bounds__(FT, 1) k_spec_cluster(const __grid_constant__ SpecArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) float2 sm[];
    float2* A = sm + OFF_A;
    float2* B = sm + OFF_B;
    float2* WH = sm + OFF_WH;
    float2* WL = sm + OFF_WL;
    uint32_t* u32 = reinterpret_cast<uint32_t*>(sm + OFF_U32);
    __shared__ float s_mu[2];
    const int r = (int)cl.block_rank();
    const int b = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t tsM = a.twM / MF;            // W_M^t = tw[t tsM]
    const int64_t tsN = a.twM / (2 * MF);      // exp(-2 pi i k / nfft) = tw[k tsN]
    const int64_t ts8 = a.twM / N2;
    for (int i = tid; i < 128; i += FT) WH[i] = a.tw[(int64_t)(64 * i) * ts8];
    for (int i = tid; i < 64; i += FT) WL[i] = a.tw[(int64_t)i * ts8];
    if (tid == 0) {
        // mean = sum / N_v in FP64 once, split as integer + fraction
        const double mu = (double)a.sums[b] / (double)a.nv;
        const double mi = rint(mu);
        s_mu[0] = (float)mi;
        s_mu[1] = (float)(mu - mi);
    }
    cl.sync();  // every CTA of the cluster has started: distributed shared memory may be used
    const float mu_i = s_mu[0], mu_f = s_mu[1];

    // ---- A: 16-point DFTs of column n2, twiddle, scatter to row k1 ----
    {
        const float* y = a.series + (int64_t)b * a.series_stride;
        const int n2 = (N2 / CL) * r + tid;
        float2 x[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) {
            const int64_t n = (int64_t)n1 * N2 + n2;
            float2 v = make_float2(0.f, 0.f);
            if (2 * n + 1 < a.nv) {
                const float2 s = *reinterpret_cast<const float2*>(y + 2 * n);
                v = make_float2((s.x - mu_i) - mu_f, (s.y - mu_i) - mu_f);
            } else if (2 * n < a.nv) {
                v.x = (y[2 * n] - mu_i) - mu_f;
            }
            x[n1] = v;
        }
        dft16(x);
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) {
            float2 v = x[k1];
            if (k1 && n2) v = cmul(v, a.tw[(int64_t)(n2 * k1) * tsM]);
            float2* Bk = cl.map_shared_rank(B, k1);
            Bk[fp(n2)] = v;
        }
    }
    cl.sync();

    // ---- B: the row's 8192-point FFT ----
    substage8192<8, 1>(B, WH, WL);
    substage8192<8, 8>(B, WH, WL);
    substage8192<8, 64>(B, WH, WL);
    substage8192<8, 512>(B, WH, WL);
    substage8192<2, 4096>(B, WH, WL);
    cl.sync();

    // ---- C: contiguous bins k = 8192 r + u: X[k1 + 16 k2] is row k1's element k2 ----
#pragma unroll 4
    for (int e = 0; e < N2 / FT; ++e) {
        const int u = tid + FT * e;
        const int k1 = u & 15, k2 = (N2 / CL) * r + (u >> 4);
        const float2* Bk = cl.map_shared_rank(B, k1);
        A[u] = Bk[fp(k2)];
    }
    cl.sync();

    // ---- D: R2C (mirror from CTA 15 - r), then whitening of 8 blocks ----
#pragma unroll 4
    for (int e = 0; e < N2 / FT; ++e) {
        const int u = tid + FT * e;
        const int64_t k = (int64_t)N2 * r + u;
        const int m = (int)((MF - k) & (MF - 1));
        const float2* Am = cl.map_shared_rank(A, m / N2);
        B[u] = r2c_bin(A[u], Am[m % N2], a.tw[k * tsN], k);
    }
    __syncthreads();
    if (warp < NW) {
        float2 v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = B[1024 * warp + lane + 32 * i];
        const int64_t k0 = (int64_t)N2 * r + 1024 * warp;
        whiten_block<32>(v, k0, lane, k0 == 0 ? 1023 : 1024, u32 + warp * NBIN, u32 + NW * NBIN + warp * NCAND,
                         u32 + NW * NBIN + NW * NCAND + warp * NCAND, 1, nullptr, B + 1024 * warp);
    }
    cl.sync();  // whitened slices of all CTAs final; the mirror reads of A are done

    // ---- E: FIR tile with halos (15 bins from CTA r-1, 16 from CTA r+1) ----
    for (int i = tid; i < TILE; i += FT) {
        const int idx = i - (NTAP / 2 - 1);
        float2 v;
        if (idx < 0) v = r == 0 ? make_float2(0.f, 0.f) : cl.map_shared_rank(B, r - 1)[N2 + idx];
        else if (idx >= N2) v = r == CL - 1 ? make_float2(0.f, 0.f) : cl.map_shared_rank(B, r + 1)[idx - N2];
        else v = B[idx];
        A[tp(i)] = v;
    }
    cl.sync();  // the neighbours' halos are read: no CTA's shared memory is used remotely after this
    {
        const float s1 = *a.tap_scale1;
        float re[RUN], im[RUN], p0[RUN];
#pragma unroll
        for (int i = 0; i < RUN; ++i) re[i] = im[i] = p0[i] = 0.f;
        const float2* w = A + tid * (RUN + RUN / 16);  // tp(RUN * tid) = 17 tid
#pragma unroll
        for (int j = 0; j < RUN + NTAP - 1; ++j) {
            const float2 xv = w[j + (j >> 4)];
#pragma unroll
            for (int i = 0; i < RUN; ++i) {
                const int ti = j - i;
                if (ti >= 0 && ti < NTAP) {
                    re[i] = fmaf(xv.x, z0_tap<NTAP>(ti), re[i]);
                    im[i] = fmaf(xv.y, z0_tap<NTAP>(ti), im[i]);
                }
                if (ti == NTAP / 2 - 1) p0[i] = pow2(xv);
            }
        }
        float2* P = reinterpret_cast<float2*>(a.plane + (int64_t)b * a.plane_stride);
        const int64_t kb = (int64_t)N2 * r + RUN * tid;
#pragma unroll
        for (int i = 0; i < RUN; ++i) {
            const float rr = re[i] * s1, qq = im[i] * s1;
            P[kb + i] = make_float2(p0[i], pow2(rr, qq));
        }
    }
}

}  // namespace

bool spec_cluster_usable() {
    static int ok = -1;  // per process: every GPU of a process is the same model here
    if (ok >= 0) return ok == 1;
    int dev = 0, v = 0;
    ok = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrClusterLaunch, dev) != cudaSuccess || !v) {
        cudaGetLastError();
        return false;
    }
    if (allow_smem((const void*)k_spec_cluster, SMEM_BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(k_spec_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(FT, 1, 1);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, (const void*)k_spec_cluster, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    ok = nclusters > 0 ? 1 : 0;
    return ok == 1;
}

cudaError_t launch_spec_cluster(const SpecArgs& a, cudaStream_t s) {
    if (a.nfft != 2 * MF || !spec_cluster_usable()) return cudaErrorInvalidValue;
    if (a.twM % (2 * MF) != 0) return cudaErrorInvalidValue;
    cudaError_t e = allow_smem((const void*)k_spec_cluster, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_spec_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, (unsigned)a.nb, 1);
    cfg.blockDim = dim3(FT, 1, 1);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_spec_cluster, a);
}

}  // namespace pss
