// f-fdot power plane (the paper's accelsearch with zmax, Sect. 3.2):
//   P[j][h] = |A(h/2, z_j)|^2,
//   A(r, z) = sum_{k=floor(r)-m+1}^{floor(r)+m} A'_k conj(rho(r - k, z)) / sqrt(E),
// z_j = -zmax + j dz, m(z) = ceil(|z|/2) + extra, E = the energy of the 2m taps.
//
// Templates: one CTA per (row, parity) evaluates conj(rho(parity/2 - t, z))
// for t = -m+1..m in FP64 (response.cuh) and stores them as FP32 together
// with 1/sqrt(E).  They depend only on (zmax, dz, extra) and are cached by
// the context.
//
// Plane: one CTA per (tile of KB bins, row, trial) stages the spectrum tile
// with its +-m halo and the row's taps in shared memory and correlates.  For
// the z = 0 row the even half-bins are |A'_k|^2 exactly and the odd ones use
// the purely imaginary sinc taps, i.e. a real-weight FIR.
#include "pss_internal.h"
#include "response.cuh"

namespace pss {

namespace {

constexpr int KB = 1024;  // bins per CTA
constexpr int NT = 256;

__global__ void k_templates(TemplateArgs a) {
    const int row = blockIdx.x >> 1, par = blockIdx.x & 1;
    const double z = -(double)a.zmax + (double)row * a.dz;
    const int m = a.tap_m[row];
    float2* out = a.taps + a.tap_off[blockIdx.x];
    double e = 0.0;
    for (int i = threadIdx.x; i < 2 * m; i += blockDim.x) {
        const int t = i - m + 1;
        const cplx r = rho_resp(0.5 * par - (double)t, z);
        out[i] = make_float2((float)r.re, (float)(-r.im));
        e += r.re * r.re + r.im * r.im;
    }
    __shared__ double red[256];
    red[threadIdx.x] = e;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.tap_scale[blockIdx.x] = (float)(1.0 / sqrt(red[0]));
}

__global__ void __launch_bounds__(NT) k_plane(PlaneArgs a) {
    extern __shared__ float2 sh[];
    const int row = blockIdx.y;
    const int b = blockIdx.z;
    const int64_t M = a.nfft / 2;
    const int64_t k0 = (int64_t)blockIdx.x * KB;
    const int m = a.tap_m[row];
    const bool z0 = (a.zmax == 0) || (-(double)a.zmax + (double)row * a.dz == 0.0);
    const float2* Ap = a.spec + (int64_t)b * a.spec_stride;
    float* P = a.plane + (int64_t)b * a.plane_stride + (int64_t)row * a.nfft;

    float2* tile = sh;                    // [KB + 2m - 1]
    float2* g0 = sh + KB + 2 * m - 1;     // [2m] parity 0 taps
    float2* g1 = g0 + 2 * m;              // [2m] parity 1 taps
    const int tw = KB + 2 * m - 1;
    for (int i = threadIdx.x; i < tw; i += NT) {
        const int64_t k = k0 - m + 1 + i;
        tile[i] = (k >= 0 && k < M) ? Ap[k] : make_float2(0.f, 0.f);
    }
    const float2* T0 = a.taps + a.tap_off[2 * row];
    const float2* T1 = a.taps + a.tap_off[2 * row + 1];
    for (int i = threadIdx.x; i < 2 * m; i += NT) {
        g0[i] = T0[i];
        g1[i] = T1[i];
    }
    __syncthreads();
    const float s0 = a.tap_scale[2 * row], s1 = a.tap_scale[2 * row + 1];
    for (int kk = threadIdx.x; kk < KB; kk += NT) {
        const int64_t k = k0 + kk;
        if (k >= M) break;
        const float2* w = tile + kk;  // w[t + m - 1] = A'[k + t]
        float p0, p1;
        if (z0) {
            const float2 c = w[m - 1];
            p0 = c.x * c.x + c.y * c.y;
            float re = 0.f, im = 0.f;
            for (int i = 0; i < 2 * m; ++i) {
                const float gy = g1[i].y;
                re = fmaf(w[i].x, gy, re);
                im = fmaf(w[i].y, gy, im);
            }
            re *= s1;
            im *= s1;
            p1 = re * re + im * im;
        } else {
            float r0 = 0.f, i0 = 0.f, r1 = 0.f, i1 = 0.f;
            for (int i = 0; i < 2 * m; ++i) {
                const float2 x = w[i];
                const float2 u = g0[i], v = g1[i];
                r0 = fmaf(x.x, u.x, r0);
                r0 = fmaf(-x.y, u.y, r0);
                i0 = fmaf(x.x, u.y, i0);
                i0 = fmaf(x.y, u.x, i0);
                r1 = fmaf(x.x, v.x, r1);
                r1 = fmaf(-x.y, v.y, r1);
                i1 = fmaf(x.x, v.y, i1);
                i1 = fmaf(x.y, v.x, i1);
            }
            r0 *= s0; i0 *= s0; r1 *= s1; i1 *= s1;
            p0 = r0 * r0 + i0 * i0;
            p1 = r1 * r1 + i1 * i1;
        }
        reinterpret_cast<float2*>(P)[k] = make_float2(p0, p1);
    }
}

// Odd half-bin tap i of the z = 0 template with 2m = NTAP taps: the
// imaginary part of conj(rho(1/2 - t, 0)) with t = i - (m - 1), which is
// 1 / (pi (t - 1/2)) (its real part is zero), rounded to FP32 at compile time.
template <int NTAP>
__host__ __device__ constexpr float z0_tap(int i) {
    return (float)(1.0 / (3.14159265358979323846 * ((double)(i - (NTAP / 2 - 1)) - 0.5)));
}

// zmax = 0 plane with 2m = NTAP taps: each thread computes R consecutive
// bins from a register window over a shared-memory tile (one padding slot
// every 8 entries keeps the strided 8-byte reads free of bank conflicts);
// the taps are compile-time constants.  Same arithmetic and order per
// output as k_plane's z = 0 rows.
template <int NTAP, int R>
__global__ void __launch_bounds__(NT) k_plane_z0(PlaneArgs a) {
    constexpr int KB0 = NT * R;
    constexpr int H = NTAP / 2 - 1;  // taps t = -H .. H+1 around the bin
    constexpr int TW = KB0 + NTAP - 1;
    __shared__ float2 tile[TW + TW / 8 + 1];
    const int b = blockIdx.y;
    const int64_t M = a.nfft / 2;
    const int64_t k0 = (int64_t)blockIdx.x * KB0;
    const float2* Ap = a.spec + (int64_t)b * a.spec_stride;
    for (int i = threadIdx.x; i < TW; i += NT) {
        const int64_t k = k0 - H + i;
        tile[i + (i >> 3)] = (k >= 0 && k < M) ? Ap[k] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float s1 = a.tap_scale[1];
    float re[R], im[R], p0[R];
#pragma unroll
    for (int i = 0; i < R; ++i) re[i] = im[i] = p0[i] = 0.f;
    const float2* w = tile + threadIdx.x * (R + R / 8);
#pragma unroll
    for (int j = 0; j < R + NTAP - 1; ++j) {
        const float2 x = w[j + (j >> 3)];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int ti = j - i;
            if (ti >= 0 && ti < NTAP) {
                re[i] = fmaf(x.x, z0_tap<NTAP>(ti), re[i]);
                im[i] = fmaf(x.y, z0_tap<NTAP>(ti), im[i]);
            }
            if (ti == H) p0[i] = x.x * x.x + x.y * x.y;
        }
    }
    float2* P = reinterpret_cast<float2*>(a.plane + (int64_t)b * a.plane_stride);
    const int64_t kb = k0 + (int64_t)threadIdx.x * R;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const float r = re[i] * s1, q = im[i] * s1;
        if (kb + i < M) P[kb + i] = make_float2(p0[i], r * r + q * q);
    }
}

}  // namespace

cudaError_t launch_templates(const TemplateArgs& a, cudaStream_t s) {
    k_templates<<<a.nz * 2, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_plane(const PlaneArgs& a, cudaStream_t s) {
    const int64_t M = a.nfft / 2;
    if (a.zmax == 0 && a.extra == 16) {
        constexpr int R = 8;
        dim3 grid((unsigned)((M + NT * R - 1) / (NT * R)), (unsigned)a.nb);
        k_plane_z0<32, R><<<grid, NT, 0, s>>>(a);
        return cudaGetLastError();
    }
    const int nz = a.zmax ? (int)llround(2.0 * a.zmax / a.dz) + 1 : 1;
    const int mmax = (int)ceil(a.zmax / 2.0) + a.extra;
    const size_t shm = (size_t)(KB + 2 * mmax - 1 + 4 * mmax) * sizeof(float2);
    {
        cudaError_t e = allow_smem((const void*)k_plane, shm);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)((M + KB - 1) / KB), (unsigned)nz, (unsigned)a.nb);
    k_plane<<<grid, NT, shm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pss
