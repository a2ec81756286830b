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
// Plane, direct form: one CTA per (tile of KB bins, row, trial) stages the
// spectrum tile with its +-m halo and the row's taps in shared memory and
// correlates.  For the z = 0 row the even half-bins are |A'_k|^2 exactly and
// the odd ones use the purely imaginary sinc taps, i.e. a real-weight FIR.
//
// Plane, overlap-save form (zmax > 0): the correlation of a row is a
// convolution of the spectrum with that row's taps, so it is done with
// L-point FFTs: a CTA transforms one segment of L spectrum bins once, then
// for every (row, parity) multiplies by the FFT of the taps, transforms back
// and keeps the L - 2 m_max + 1 outputs that the circular wrap does not
// touch.  About 70 flops per plane value instead of 16 m(z).
#include <stdlib.h>

#include "bulk.cuh"
#include "fft_small.cuh"
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
            p0 = pow2(c);
            float re = 0.f, im = 0.f;
            for (int i = 0; i < 2 * m; ++i) {
                const float gy = g1[i].y;
                re = fmaf(w[i].x, gy, re);
                im = fmaf(w[i].y, gy, im);
            }
            re *= s1;
            im *= s1;
            p1 = pow2(re, im);
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
            p0 = pow2(r0, i0);
            p1 = pow2(r1, i1);
        }
        reinterpret_cast<float2*>(P)[k] = make_float2(p0, p1);
    }
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
            if (ti == H) p0[i] = pow2(x);
        }
    }
    float2* P = reinterpret_cast<float2*>(a.plane + (int64_t)b * a.plane_stride);
    const int64_t kb = k0 + (int64_t)threadIdx.x * R;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const float r = re[i] * s1, q = im[i] * s1;
        if (kb + i < M) P[kb + i] = make_float2(p0[i], pow2(r, q));
    }
}

// The same FIR, double-buffered: a CTA walks `tpc` consecutive tiles of one
// trial and brings tile t+1 into a second shared-memory buffer by
// asynchronous 8-byte copies (zero-filled outside the spectrum) while it
// computes tile t.  Same arithmetic and order: bit-identical planes.
template <int NTAP, int R>
__global__ void __launch_bounds__(NT) k_plane_z0_db(PlaneArgs a, int tpc) {
    constexpr int KB0 = NT * R;
    constexpr int H = NTAP / 2 - 1;
    constexpr int TW = KB0 + NTAP - 1;
    constexpr int TWP = TW + TW / 8 + 1;
    __shared__ float2 tiles[2 * TWP];
    const int b = blockIdx.y;
    const int64_t M = a.nfft / 2;
    const int64_t ntile = (M + KB0 - 1) / KB0;
    const int64_t tile0 = (int64_t)blockIdx.x * tpc;
    const int64_t tile1 = min(ntile, tile0 + tpc);
    const float2* Ap = a.spec + (int64_t)b * a.spec_stride;
    auto issue = [&](int64_t tt, float2* buf) {
        const int64_t k0 = tt * KB0;
        for (int i = threadIdx.x; i < TW; i += NT) {
            const int64_t k = k0 - H + i;
            const bool ok = k >= 0 && k < M;
            cp_async8(buf + i + (i >> 3), ok ? (const void*)(Ap + k) : (const void*)Ap, ok ? 8u : 0u);
        }
    };
    issue(tile0, tiles);
    cp_async_commit();
    const float s1 = a.tap_scale[1];
    float2* P = reinterpret_cast<float2*>(a.plane + (int64_t)b * a.plane_stride);
    for (int64_t t = tile0; t < tile1; ++t) {
        const float2* cur = tiles + ((t - tile0) & 1) * TWP;
        if (t + 1 < tile1) {
            issue(t + 1, tiles + ((t + 1 - tile0) & 1) * TWP);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        float re[R], im[R], p0[R];
#pragma unroll
        for (int i = 0; i < R; ++i) re[i] = im[i] = p0[i] = 0.f;
        const float2* w = cur + threadIdx.x * (R + R / 8);
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
                if (ti == H) p0[i] = pow2(x);
            }
        }
        const int64_t kb = t * KB0 + (int64_t)threadIdx.x * R;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const float r = re[i] * s1, q = im[i] * s1;
            if (kb + i < M) P[kb + i] = make_float2(p0[i], pow2(r, q));
        }
        __syncthreads();
    }
}

// PSS_PLANE_Z0_DB=0 keeps the single-buffered zmax 0 plane; PSS_PLANE_Z0_TPC
// sets the tiles per CTA of the double-buffered one (default 4).
int plane_z0_tpc() {
    static const int v = [] {
        const char* e = getenv("PSS_PLANE_Z0_DB");
        if (e && e[0] == '0') return 0;
        const char* t = getenv("PSS_PLANE_Z0_TPC");
        const int x = t ? atoi(t) : 4;
        return x < 1 ? 1 : x;
    }();
    return v;
}

// ---- overlap-save plane ------------------------------------------------------

// Template spectra, FP64: for row z_j and parity p the taps
// g[t] = conj(rho(p/2 - t, z_j)), t = -m+1..m, sit at circular position
// s = t + M0 (M0 = m_max - 1), and
//   T[f] = (1 / (L sqrt(E))) sum_t g[t] exp(+2 pi i f s / L),
// so that FFT(conj(X T)) of a segment's spectrum X is conj(L) times the
// circular correlation with g / sqrt(E): its squared magnitude at u is the
// plane value of the segment's u-th valid bin.  One CTA per (row, parity).
__global__ void k_fft_templates(FftTemplateArgs a) {
    extern __shared__ double2 fts[];
    double2* g = fts;              // [2 m]
    double2* W = fts + 2 * 1024;   // [L] exp(+2 pi i n / L)
    __shared__ double red[256];
    const int row = blockIdx.x >> 1, par = blockIdx.x & 1;
    const double z = -(double)a.zmax + (double)row * a.dz;
    const int m = a.tap_m[row];
    double e = 0.0;
    for (int i = threadIdx.x; i < 2 * m; i += blockDim.x) {
        const int t = i - m + 1;
        const cplx r = rho_resp(0.5 * par - (double)t, z);
        g[i] = make_double2(r.re, -r.im);
        e += r.re * r.re + r.im * r.im;
    }
    for (int n = threadIdx.x; n < a.L; n += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)n / (double)a.L, &sn, &cs);
        W[n] = make_double2(cs, sn);
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    const double scale = 1.0 / ((double)a.L * sqrt(red[0]));
    float2* out = a.ftaps + (int64_t)blockIdx.x * a.L;
    for (int f = threadIdx.x; f < a.L; f += blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int i = 0; i < 2 * m; ++i) {
            const int s = i - m + 1 + a.M0;  // 0 <= s < L
            const double2 w = W[(f * s) & (a.L - 1)];  // L is a power of two
            re += g[i].x * w.x - g[i].y * w.y;
            im += g[i].x * w.y + g[i].y * w.x;
        }
        out[f] = make_float2((float)(re * scale), (float)(im * scale));
    }
}

constexpr int FNT = 256;

// Twiddles of the sub-stages with running span NS: table [q][k] =
// exp(-2 pi i q k / (RR NS)) (q-major, so lanes with consecutive k read
// consecutive words).  Offsets of the three tables of L = 2048 = 8*8*8*4.
constexpr int TW2 = 0;            // RR 8, NS 8:   8 x 8
constexpr int TW3 = TW2 + 64;     // RR 8, NS 64:  8 x 64
constexpr int TW4 = TW3 + 512;    // RR 4, NS 512: 4 x 512
constexpr int TWN = TW4 + 2048;

// One in-place Stockham sub-stage of radix RR and running span NS of two
// L-point forward FFTs held in shared memory (natural order in and out after
// all sub-stages); each thread runs the same butterflies on both.
template <int L, int RR, int NS>
__device__ __forceinline__ void fft_substage2(float2* b0, float2* b1, const float2* twt) {
    constexpr int NB = L / RR;
    constexpr int PER = NB / FNT;
    float2 x0[PER][RR], x1[PER][RR];
    int dst[PER];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * FNT;
        const int k = b & (NS - 1);
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            x0[p][q] = b0[fp(b + q * NB)];
            x1[p][q] = b1[fp(b + q * NB)];
            if (NS > 1 && q) {
                const float2 w = twt[q * NS + k];
                x0[p][q] = cmul(x0[p][q], w);
                x1[p][q] = cmul(x1[p][q], w);
            }
        }
        dst[p] = (b - k) * RR + k;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        dft_small<RR>(x0[p]);
        dft_small<RR>(x1[p]);
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            b0[fp(dst[p] + q * NS)] = x0[p][q];
            b1[fp(dst[p] + q * NS)] = x1[p][q];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void fft2048x2(float2* b0, float2* b1, const float2* twt) {
    fft_substage2<2048, 8, 1>(b0, b1, twt);
    fft_substage2<2048, 8, 8>(b0, b1, twt + TW2);
    fft_substage2<2048, 8, 64>(b0, b1, twt + TW3);
    fft_substage2<2048, 4, 512>(b0, b1, twt + TW4);
}

__global__ void __launch_bounds__(FNT, 3) k_plane_fft(const __grid_constant__ PlaneArgs a) {
    constexpr int L = PLANE_FFT_L;
    static_assert(L == 2048, "sub-stage tables are laid out for 2048 points");
    constexpr int PADL = L;
    constexpr int NE = L / FNT;
    extern __shared__ float2 fsm[];
    float2* Y0 = fsm;             // work, parity 0 (first: the segment)
    float2* Y1 = fsm + PADL;      // work, parity 1
    float2* twt = fsm + 2 * PADL;
    const int b = blockIdx.y;
    const int64_t M = a.nfft / 2;
    const int V = a.fV, M0 = a.fM0;
    const int64_t k0 = (int64_t)blockIdx.x * V;
    const float2* Ap = a.spec + (int64_t)b * a.spec_stride;
    const int64_t tstride = a.twM / L;  // global table: exp(-2 pi i t / twM)
    for (int i = threadIdx.x; i < TWN; i += FNT) {
        int rr, ns, o;
        if (i < TW3) { rr = 8; ns = 8; o = i - TW2; }
        else if (i < TW4) { rr = 8; ns = 64; o = i - TW3; }
        else { rr = 4; ns = 512; o = i - TW4; }
        const int q = o / ns, k = o - q * ns;
        twt[i] = a.tw[(int64_t)(q * k * (L / (rr * ns))) * tstride];
    }
    for (int i = threadIdx.x; i < L; i += FNT) {
        const int64_t k = k0 - M0 + i;
        Y0[fp(i)] = (k >= 0 && k < M) ? Ap[k] : make_float2(0.f, 0.f);
        Y1[fp(i)] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft2048x2(Y0, Y1, twt);  // the segment's spectrum (the second transform is idle)
    float2 X[NE];            // each thread keeps the bins it multiplies
#pragma unroll
    for (int e = 0; e < NE; ++e) X[e] = Y0[fp(threadIdx.x + e * FNT)];
    __syncthreads();
    const int nz = a.nz;
    float2* P = reinterpret_cast<float2*>(a.plane + (int64_t)b * a.plane_stride);
    for (int j = 0; j < nz; ++j) {
        const bool zrow0 = (j == a.zrow0);
        const float2* T0 = a.ftaps + (int64_t)j * 2 * L;
        const float2* T1 = T0 + L;
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int i = threadIdx.x + e * FNT;
            const float2 y0 = cmul(X[e], __ldg(T0 + i)), y1 = cmul(X[e], __ldg(T1 + i));
            Y0[fp(i)] = make_float2(y0.x, -y0.y);
            Y1[fp(i)] = make_float2(y1.x, -y1.y);
        }
        __syncthreads();
        fft2048x2(Y0, Y1, twt);
        float2* row = P + (int64_t)j * M;
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            const int u = threadIdx.x + e * FNT;
            const int64_t k = k0 + u;
            if (u < V && k < M) {
                const float2 y0 = Y0[fp(u)], y1 = Y1[fp(u)];
                float p0 = pow2(y0);
                if (zrow0) {
                    // integer half-bins of the z = 0 row: the raw powers, exactly
                    const float2 c = Ap[k];
                    p0 = pow2(c);
                }
                row[k] = make_float2(p0, pow2(y1));
            }
        }
        __syncthreads();
    }
}

// ---- overlap-save plane, radix 16-16-8 form (an autotuner choice) -------------------
// The same correlation as k_plane_fft with 128 threads and three in-place
// sub-stages (radix 16, 16, 8) instead of four: fewer shared-memory passes
// and barriers per row, at lower thread count.
constexpr int F16NT = 128;
constexpr int T16A = 0;             // RR 16, NS 16: 16 x 16
constexpr int T16B = T16A + 256;    // RR 8, NS 256: 8 x 256
constexpr int T16N = T16B + 2048;

template <int RR, int NS>
__device__ __forceinline__ void fft16_substage2(float2* b0, float2* b1, const float2* twt) {
    constexpr int L = PLANE_FFT_L;
    constexpr int NB = L / RR;
    constexpr int PER = NB / F16NT;
    float2 x0[PER][RR], x1[PER][RR];
    int dst[PER];
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int b = threadIdx.x + p * F16NT;
        const int k = b & (NS - 1);
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            x0[p][q] = b0[fx(b + q * NB)];
            x1[p][q] = b1[fx(b + q * NB)];
            if (NS > 1 && q) {
                const float2 w = twt[q * NS + k];
                x0[p][q] = cmul(x0[p][q], w);
                x1[p][q] = cmul(x1[p][q], w);
            }
        }
        dst[p] = (b - k) * RR + k;
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        dft_any<RR>(x0[p]);
        dft_any<RR>(x1[p]);
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            b0[fx(dst[p] + q * NS)] = x0[p][q];
            b1[fx(dst[p] + q * NS)] = x1[p][q];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void fft2048x2_r16(float2* b0, float2* b1, const float2* twt) {
    fft16_substage2<16, 1>(b0, b1, twt);
    fft16_substage2<16, 16>(b0, b1, twt + T16A);
    fft16_substage2<8, 256>(b0, b1, twt + T16B);
}

__global__ void __launch_bounds__(F16NT, 4) k_plane_fft16(const __grid_constant__ PlaneArgs a) {
    constexpr int L = PLANE_FFT_L;
    constexpr int NE = L / F16NT;  // 16 bins per thread
    extern __shared__ float2 fsm[];
    float2* Y0 = fsm;
    float2* Y1 = fsm + L;
    float2* twt = fsm + 2 * L;
    const int b = blockIdx.y;
    const int64_t M = a.nfft / 2;
    const int V = a.fV, M0 = a.fM0;
    const int64_t k0 = (int64_t)blockIdx.x * V;
    const float2* Ap = a.spec + (int64_t)b * a.spec_stride;
    const int64_t tstride = a.twM / L;
    for (int i = threadIdx.x; i < T16N; i += F16NT) {
        int rr, ns, o;
        if (i < T16B) { rr = 16; ns = 16; o = i - T16A; }
        else { rr = 8; ns = 256; o = i - T16B; }
        const int q = o / ns, k = o - q * ns;
        twt[i] = a.tw[(int64_t)(q * k * (L / (rr * ns))) * tstride];
    }
    for (int i = threadIdx.x; i < L; i += F16NT) {
        const int64_t k = k0 - M0 + i;
        Y0[fx(i)] = (k >= 0 && k < M) ? Ap[k] : make_float2(0.f, 0.f);
        Y1[fx(i)] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft2048x2_r16(Y0, Y1, twt);
    float2 X[NE];
#pragma unroll
    for (int e = 0; e < NE; ++e) X[e] = Y0[fx(threadIdx.x + e * F16NT)];
    __syncthreads();
    const int nz = a.nz;
    float2* P = reinterpret_cast<float2*>(a.plane + (int64_t)b * a.plane_stride);
    // Per row: the first radix-16 sub-stage (running span 1) takes butterfly b = thread's
    // elements b + 128 q, which are the thread's own bins X[q]: it runs on the products in
    // registers; the middle sub-stage runs in shared memory; the last (radix 8, span 256)
    // reads its inputs and writes the powers of its outputs b + 256 q straight to the plane.
    // The same operations in the same order as the in-place form (bit-identical output).
    for (int j = 0; j < nz; ++j) {
        const bool zrow0 = (j == a.zrow0);
        const float2* T0 = a.ftaps + (int64_t)j * 2 * L;
        const float2* T1 = T0 + L;
        {
            float2 x0[NE], x1[NE];
#pragma unroll
            for (int e = 0; e < NE; ++e) {
                const int i = threadIdx.x + e * F16NT;
                const float2 y0 = cmul(X[e], __ldg(T0 + i)), y1 = cmul(X[e], __ldg(T1 + i));
                x0[e] = make_float2(y0.x, -y0.y);
                x1[e] = make_float2(y1.x, -y1.y);
            }
            dft_any<16>(x0);
            dft_any<16>(x1);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                Y0[fx(threadIdx.x * 16 + q)] = x0[q];
                Y1[fx(threadIdx.x * 16 + q)] = x1[q];
            }
        }
        __syncthreads();
        fft16_substage2<16, 16>(Y0, Y1, twt + T16A);
        float2* row = P + (int64_t)j * M;
        {
            constexpr int NS = 256, NB = L / 8, PER = NB / F16NT;
            const float2* tl = twt + T16B;
#pragma unroll
            for (int p = 0; p < PER; ++p) {
                const int bb = threadIdx.x + p * F16NT;  // < NS: its span index k is bb itself
                float2 x0[8], x1[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    x0[q] = Y0[fx(bb + q * NB)];
                    x1[q] = Y1[fx(bb + q * NB)];
                    if (q) {
                        const float2 w = tl[q * NS + bb];
                        x0[q] = cmul(x0[q], w);
                        x1[q] = cmul(x1[q], w);
                    }
                }
                dft_any<8>(x0);
                dft_any<8>(x1);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int u = bb + q * NS;
                    const int64_t k = k0 + u;
                    if (u < V && k < M) {
                        float p0 = pow2(x0[q]);
                        if (zrow0) {
                            const float2 c = Ap[k];
                            p0 = pow2(c);
                        }
                        row[k] = make_float2(p0, pow2(x1[q]));
                    }
                }
            }
        }
        __syncthreads();  // the next row's first sub-stage overwrites Y0 / Y1
    }
}

}  // namespace

cudaError_t launch_fft_templates(const FftTemplateArgs& a, cudaStream_t s) {
    if (a.L != PLANE_FFT_L) return cudaErrorInvalidValue;
    const size_t shm = (size_t)(2 * 1024 + a.L) * sizeof(double2);
    cudaError_t e = allow_smem((const void*)k_fft_templates, shm);
    if (e != cudaSuccess) return e;
    k_fft_templates<<<a.nz * 2, 256, shm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_templates(const TemplateArgs& a, cudaStream_t s) {
    k_templates<<<a.nz * 2, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_plane(const PlaneArgs& a, cudaStream_t s) {
    const int64_t M = a.nfft / 2;
    if (a.zmax == 0 && a.extra == 16) {
        constexpr int R = 8;
        const int64_t ntile = (M + NT * R - 1) / (NT * R);
        const int tpc = plane_z0_tpc();
        if (tpc > 0) {
            const int64_t per = std::min<int64_t>(tpc, ntile);
            dim3 grid((unsigned)((ntile + per - 1) / per), (unsigned)a.nb);
            k_plane_z0_db<32, R><<<grid, NT, 0, s>>>(a, (int)per);
            return cudaGetLastError();
        }
        dim3 grid((unsigned)ntile, (unsigned)a.nb);
        k_plane_z0<32, R><<<grid, NT, 0, s>>>(a);
        return cudaGetLastError();
    }
    const int nz = a.zmax ? (int)llround(2.0 * a.zmax / a.dz) + 1 : 1;
    if (a.ftaps && a.form == 1) {
        if (a.fL != PLANE_FFT_L || a.fV <= 0 || a.twM % PLANE_FFT_L) return cudaErrorInvalidValue;
        const size_t shm = (size_t)(2 * PLANE_FFT_L + T16N) * sizeof(float2);
        cudaError_t e = allow_smem((const void*)k_plane_fft16, shm);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((M + a.fV - 1) / a.fV), (unsigned)a.nb);
        k_plane_fft16<<<grid, F16NT, shm, s>>>(a);
        return cudaGetLastError();
    }
    if (a.ftaps) {
        if (a.fL != PLANE_FFT_L || a.fV <= 0 || a.twM % PLANE_FFT_L) return cudaErrorInvalidValue;
        const size_t shm = (size_t)(2 * PLANE_FFT_L + TWN) * sizeof(float2);
        cudaError_t e = allow_smem((const void*)k_plane_fft, shm);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((M + a.fV - 1) / a.fV), (unsigned)a.nb);
        k_plane_fft<<<grid, FNT, shm, s>>>(a);
        return cudaGetLastError();
    }
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
