// Small forward DFTs in registers (lengths 2, 4, 8) and complex helpers,
// shared by the batched FFT passes and the overlap-save plane kernel.
//   x[k] = sum_n x[n] exp(-2 pi i n k / L)
#pragma once
#include <cuda_runtime.h>

namespace pss {

constexpr float R2 = 0.70710678118654752440f;  // 1/sqrt(2)

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // * (-i)

// forward DFTs of length 2, 4, 8 in registers (x[k] = sum_n x[n] e^{-2 pi i nk/L})
__device__ __forceinline__ void dft2(float2* x) {
    const float2 a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
}
__device__ __forceinline__ void dft4(float2& y0, float2& y1, float2& y2, float2& y3) {
    const float2 s02 = cadd(y0, y2), d02 = csub(y0, y2);
    const float2 s13 = cadd(y1, y3), d13 = mul_mi(csub(y1, y3));
    y0 = cadd(s02, s13);
    y2 = csub(s02, s13);
    const float2 t1 = cadd(d02, d13), t3 = csub(d02, d13);
    y1 = t1;
    y3 = t3;
}
__device__ __forceinline__ void dft4v(float2* x) { dft4(x[0], x[1], x[2], x[3]); }
__device__ __forceinline__ void dft8(float2* x) {
    float2 a0 = cadd(x[0], x[4]), b0 = csub(x[0], x[4]);
    float2 a1 = cadd(x[1], x[5]), b1 = csub(x[1], x[5]);
    float2 a2 = cadd(x[2], x[6]), b2 = csub(x[2], x[6]);
    float2 a3 = cadd(x[3], x[7]), b3 = csub(x[3], x[7]);
    // b_m *= w^m, w = exp(-2 pi i / 8)
    b1 = make_float2((b1.x + b1.y) * R2, (b1.y - b1.x) * R2);
    b2 = mul_mi(b2);
    b3 = make_float2((b3.y - b3.x) * R2, -(b3.x + b3.y) * R2);
    dft4(a0, a1, a2, a3);
    dft4(b0, b1, b2, b3);
    x[0] = a0; x[2] = a1; x[4] = a2; x[6] = a3;
    x[1] = b0; x[3] = b1; x[5] = b2; x[7] = b3;
}

template <int RR>
__device__ __forceinline__ void dft_small(float2* x) {
    if constexpr (RR == 2) dft2(x);
    else if constexpr (RR == 4) dft4v(x);
    else dft8(x);
}

// W_16^m = exp(-2 pi i m / 16)
__device__ __forceinline__ float2 w16(int m) {
    constexpr float C[16] = {1.f,          0.92387953f,  0.70710678f,  0.38268343f, 0.f,          -0.38268343f,
                             -0.70710678f, -0.92387953f, -1.f,         -0.92387953f, -0.70710678f, -0.38268343f,
                             0.f,          0.38268343f,  0.70710678f,  0.92387953f};
    return make_float2(C[m & 15], -C[(m + 12) & 15]);  // (cos, -sin): sin(x) = cos(x - pi/2)
}

// 16-point forward DFT in registers (4 x 4), natural order in and out
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
    float2 y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        float2 t[4] = {x[n2], x[4 + n2], x[8 + n2], x[12 + n2]};
        dft4v(t);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) y[n2][k1] = (n2 && k1) ? cmul(t[k1], w16(n2 * k1)) : t[k1];
    }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 t[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
        dft4v(t);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) x[k1 + 4 * k2] = t[k2];
    }
}

template <int RR>
__device__ __forceinline__ void dft_any(float2 (&x)[RR]) {
    if constexpr (RR == 16) dft16(x);
    else dft_small<RR>(x);
}

// Swizzled shared-memory index for 8-byte elements: within each run of 16
// (one 128-byte line) the slot is XORed with a function of the run number,
// chosen so that every access of the 8-8-8-4 sub-stage order (16 consecutive
// elements; or 8 runs of 2 at stride 8; or 2 runs of 8 at stride 64) hits 16
// different bank pairs per half-warp.
__host__ __device__ __forceinline__ int fp(int i) {
    const int r = i >> 4;
    const int g = (r & 7) | ((r & 4) << 1);
    return (i & ~15) | ((i & 15) ^ g);
}


// A second swizzle for the 16-16-8 sub-stage order (strided writes of 16
// runs of one element, or 16 consecutive elements): the slot is XORed with
// the run number.
__host__ __device__ __forceinline__ int fx(int i) { return (i & ~15) | ((i & 15) ^ ((i >> 4) & 15)); }

// |x|^2 with a fixed rounding: x.x^2 rounded, then x.y^2 added by one fused
// multiply-add, so that every kernel forming a power gets the same bits
// whatever the compiler would otherwise contract.
__device__ __forceinline__ float pow2(float2 x) { return fmaf(x.y, x.y, __fmul_rn(x.x, x.x)); }
__device__ __forceinline__ float pow2(float re, float im) { return fmaf(im, im, __fmul_rn(re, re)); }

// Odd half-bin tap i of the z = 0 template with 2m = NTAP taps: the
// imaginary part of conj(rho(1/2 - t, 0)) with t = i - (m - 1), which is
// 1 / (pi (t - 1/2)) (its real part is zero), rounded to FP32 at compile time.
template <int NTAP>
__host__ __device__ constexpr float z0_tap(int i) {
    return (float)(1.0 / (3.14159265358979323846 * ((double)(i - (NTAP / 2 - 1)) - 0.5)));
}

}  // namespace pss
