// Candidate refinement in continuous (DM, r, z): the objective, its analytic
// gradient, and the per-channel spectra it needs.  The paper folds
// candidates (prepfold, Sect. 2 step 6) and has no continuous refinement;
// the objective is this library's:
//
//   P_h(DM, r, z) = sum_{k=1..h} g(floor(kr)) |F_k|^2 / E_k,
//   F_k = sum_c exp(i phi_ck) G_ck,   G_ck = sum_q A^c_q conj(rho(kr - q, kz)),
//   phi_ck = 2 pi (k r) DM dtau_c / T,  E_k = sum_q |rho(kr - q, kz)|^2,
//
// over the 2m(kz) bins q nearest kr (bins outside [0, nfft/2) add nothing),
// A^c the mean-subtracted spectrum of channel c alone, dtau_c the
// dispersion delay per unit DM relative to the top channel (seconds), T the
// series span and g the whitening gain (ln 2 / median power) of the block
// holding floor(kr) in the candidate's own DM trial.
//
// Gradient (the tap set and g are piecewise constant and contribute none):
//   dF/dDM = sum_c i (2 pi k r dtau_c / T) e^{i phi} G_c,
//   dF/dr  = sum_c e^{i phi} (i (2 pi k DM dtau_c / T) G_c + k Gq_c),
//   dF/dz  = sum_c e^{i phi} k Gz_c,
//   Gq_c = sum_q A^c_q conj(rho_q), Gz_c = sum_q A^c_q conj(rho_z),
//   dE/dr = k sum_q 2 Re(conj(rho) rho_q), dE/dz = k sum_q 2 Re(conj(rho) rho_z),
//   dP/dx = g (2 Re(conj(F) dF/dx) / E - |F|^2 (dE/dx) / E^2).
// Phases are evaluated in FP64 (harmonic k's channel phases as the k-th
// power of the fundamental's); the response taps (rho_derivs, response.cuh)
// in FP64 for |kz| < 8 and above that with FP64 phase arguments and FP32
// magnitudes (rho_derivs_mixed);
// the phased channel sums per tap (lanes over taps, warps over channel
// groups) accumulate in FP32 and are reduced across the CTA in FP64.
#include <math.h>

#include "pss_internal.h"
#include "response.cuh"

namespace pss {

namespace {

constexpr int NT = 256;
constexpr int MAXTAP = 2 * (600 + 64);  // 2 m for |k z| <= 1200, extra <= 64

// per-channel boxcar series (ds native samples per output) and their sums
__global__ void k_chan_series(const uint8_t* xcm, int64_t pitch, int32_t ck, int64_t nv, int32_t ds, float* out,
                              int64_t out_stride, unsigned long long* sums) {
    const int c = blockIdx.y;
    const uint8_t* row = xcm + (int64_t)c * pitch;
    unsigned long long part = 0ull;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nv; j += (int64_t)gridDim.x * blockDim.x) {
        uint32_t acc = 0;
        for (int e = 0; e < ds; ++e) acc += row[j * ds + e];
        out[(int64_t)c * out_stride + j] = (float)acc;
        part += acc;
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(sums + c, part);
}

// ---- response taps for |z| >= RESP_F32_Z, FP32 with FP64 phase arguments ---
// rho and its derivatives (same formulas as rho_derivs in response.cuh) with
// every phase argument formed and reduced modulo 2 in FP64 and the rest in
// FP32.  Above |z| = 8 the integration-by-parts solve for M1, M2 divides by z
// with |q - z/2| / |z| <= 1 + extra / |z|, so FP32 errors stay near 1e-6 of
// the taps; below it the FP64 evaluation runs.
constexpr double RESP_F32_Z = 8.0;

// x mod 2 in [-1, 1], FP64, as a float (an argument for sincospif)
__device__ __forceinline__ float mod2f(double x) { return (float)(x - 2.0 * rint(0.5 * x)); }

// Fresnel C, S of x as C = sgn (1/2 + oc), S = sgn (1/2 + os), sgn = sign(x):
// the offsets from 1/2 are what a difference of two same-side values needs.
__device__ __forceinline__ void fresnel_off(double x, float* sgn, float* oc, float* os) {
    const double axd = fabs(x);
    const float ax = (float)axd;
    *sgn = x < 0 ? -1.f : 1.f;
    if (ax <= 2.f) {
        // power series (A&S 7.3.11, 7.3.13), terms (pi/2)^k x^(2k+1) / (k! (2k+1))
        float t = ax, c = 0.f, sv = 0.f;
        const float a2 = 1.5707963267948966f * ax * ax;
        for (int k = 0; k < 40; ++k) {
            const float term = t / (float)(2 * k + 1);
            switch (k & 3) {
                case 0: c += term; break;
                case 1: sv += term; break;
                case 2: c -= term; break;
                default: sv -= term; break;
            }
            t *= a2 / (float)(k + 1);
            if (t < 1e-9f) break;
        }
        *oc = c - 0.5f;
        *os = sv - 0.5f;
        return;
    }
    // continued fraction of erfc (A&S 7.1.14) for the auxiliary functions f, g
    // (forward three-term recurrences as in fresnel_cs: one division)
    const float h = 0.88622692545275801f * ax;  // sqrt(pi) / 2 * x; zeta = h (1 - i)
    int nt = (int)ceilf(220.f / (ax * ax)) + 6;
    if (nt > 60) nt = 60;
    if (ax > 1e4f) nt = 1;  // zeta^2 must stay inside the FP32 range
    float a1r = h, a1i = -h, a2r = 1.f, a2i = 0.f, b1r = 1.f, b1i = 0.f, b2r = 0.f, b2i = 0.f;
    for (int k = 1; k <= nt; ++k) {
        const float kk = 0.5f * (float)k;
        const float ar = h * a1r + h * a1i + kk * a2r, ai = h * a1i - h * a1r + kk * a2i;
        const float br = h * b1r + h * b1i + kk * b2r, bi = h * b1i - h * b1r + kk * b2i;
        a2r = a1r;
        a2i = a1i;
        a1r = ar;
        a1i = ai;
        b2r = b1r;
        b2i = b1i;
        b1r = br;
        b1i = bi;
        // A, B grow like prod (k/2): rescale both (their ratio is the value) so
        // that |A|^2 in the final division stays inside the FP32 range
        if (fabsf(a1r) + fabsf(a1i) > 1e15f) {
            a1r *= 1e-15f;
            a1i *= 1e-15f;
            a2r *= 1e-15f;
            a2i *= 1e-15f;
            b1r *= 1e-15f;
            b1i *= 1e-15f;
            b2r *= 1e-15f;
            b2i *= 1e-15f;
        }
    }
    // K = B / A
    const float den = a1r * a1r + a1i * a1i;
    const float Kr = (b1r * a1r + b1i * a1i) / den, Ki = (b1i * a1r - b1r * a1i) / den;
    const float fac = 0.28209479177387814f;  // 1 / (2 sqrt(pi))
    const float g = fac * (Kr - Ki), f = fac * (Kr + Ki);
    float sn, cs;
    sincospif(mod2f(0.5 * axd * axd), &sn, &cs);
    *oc = f * sn - g * cs;
    *os = -f * cs - g * sn;
}

__device__ __forceinline__ float2 c_mulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ void rho_derivs_mixed(double q, double z, float2* r, float2* rq, float2* rz) {
    const double sqd = sqrt(2.0 * fabs(z));
    const double bb = (q - 0.5 * z) / z;
    float g0, c0, s0, g1, c1, s1;
    fresnel_off(sqd * bb, &g0, &c0, &s0);
    fresnel_off(sqd * (1.0 + bb), &g1, &c1, &s1);
    const float isq = (float)(1.0 / sqd);
    // C(w1) - C(w0) with the halves taken exactly
    const float dC = (0.5f * (g1 - g0) + (g1 * c1 - g0 * c0)) * isq;
    const float dS = (z > 0 ? 1.f : -1.f) * (0.5f * (g1 - g0) + (g1 * s1 - g0 * s0)) * isq;
    const double qq = q - 0.5 * z;
    float sn, cs;
    sincospif(mod2f(-(qq * qq) / z), &sn, &cs);
    const float2 rho = c_mulf(make_float2(cs, sn), make_float2(dC, dS));
    float es, ec;
    sincospif(mod2f(2.0 * q), &es, &ec);
    const float af = (float)qq, zf = (float)z;
    const float i2p = 0.15915494309189535f;  // 1 / (2 pi); (x) / (2 pi i) = (x.y, -x.x) / (2 pi)
    const float2 t1 = make_float2(es * i2p, -(ec - 1.f) * i2p);
    const float2 M1 = make_float2((t1.x - af * rho.x) / zf, (t1.y - af * rho.y) / zf);
    const float2 t2 = make_float2((es - rho.y) * i2p, -(ec - rho.x) * i2p);
    const float2 M2 = make_float2((t2.x - af * M1.x) / zf, (t2.y - af * M1.y) / zf);
    *r = rho;
    *rq = make_float2(-6.283185307179586f * M1.y, 6.283185307179586f * M1.x);            // 2 pi i M1
    *rz = make_float2(-3.141592653589793f * (M2.y - M1.y), 3.141592653589793f * (M2.x - M1.x));  // pi i (M2 - M1)
}

__device__ __forceinline__ double2 block_sum2(double2 v, double* red) {
    // reduce (x, y) over the CTA; red holds 2 * NT / 32 doubles
    for (int off = 16; off > 0; off >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) {
        red[2 * w] = v.x;
        red[2 * w + 1] = v.y;
    }
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    for (int i = 0; i < NT / 32; ++i) {
        r.x += red[2 * i];
        r.y += red[2 * i + 1];
    }
    return r;
}

__global__ void __launch_bounds__(NT) k_refine_eval(const __grid_constant__ RefineArgs a) {
    __shared__ float2 s_r[MAXTAP], s_rq[MAXTAP], s_rz[MAXTAP];
    __shared__ double red[2 * NT / 32];
    extern __shared__ float4 s_ch[];  // [ck] channel phase e_c and dtau_c e_c of the harmonic
    const int p = blockIdx.x;
    const RefinePt pt = a.pts[p];
    const int64_t M = a.nfft / 2;
    double P = 0.0, gdm = 0.0, gr = 0.0, gz = 0.0;
    // channel phases exp(i 2 pi (k r) DM dtau_c / T): the fundamental's by
    // sincospi (FP64), each further harmonic by one FP64 complex product
    // (phi_ck = k phi_c1), for the CPT channels a thread owns
    constexpr int CPT = 4;
    const bool rec = a.ck <= CPT * NT;
    double e1c[CPT], e1s[CPT], ekc[CPT], eks[CPT];
#pragma unroll
    for (int i = 0; i < CPT; ++i) {
        e1c[i] = 1.0;
        e1s[i] = 0.0;
        ekc[i] = 1.0;
        eks[i] = 0.0;
        const int c = threadIdx.x + i * NT;
        if (rec && c < a.ck) sincospi(2.0 * pt.r * pt.dm * a.dtau[c] / a.T, &e1s[i], &e1c[i]);
    }
    for (int k = 1; k <= pt.numharm; ++k) {
        if (rec) {
#pragma unroll
            for (int i = 0; i < CPT; ++i) {
                const double c2 = ekc[i] * e1c[i] - eks[i] * e1s[i];
                eks[i] = ekc[i] * e1s[i] + eks[i] * e1c[i];
                ekc[i] = c2;
            }
        }
        const double rk = k * pt.r, zk = k * pt.z;
        const int m = (int)ceil(fabs(zk) / 2.0) + a.extra;
        if (2 * m > MAXTAP) break;
        const int64_t k0 = (int64_t)floor(rk);
        // taps: conj(rho), conj(rho_q), conj(rho_z); energies E, Eq, Ez
        double e0 = 0.0, eq = 0.0, ez = 0.0;
        for (int t = threadIdx.x; t < 2 * m; t += NT) {
            const int64_t q = k0 - m + 1 + t;
            if (fabs(zk) >= RESP_F32_Z) {
                float2 r, rq, rz;
                rho_derivs_mixed(rk - (double)q, zk, &r, &rq, &rz);
                s_r[t] = make_float2(r.x, -r.y);
                s_rq[t] = make_float2(rq.x, -rq.y);
                s_rz[t] = make_float2(rz.x, -rz.y);
                e0 += (double)(r.x * r.x + r.y * r.y);
                eq += (double)(2.f * (r.x * rq.x + r.y * rq.y));
                ez += (double)(2.f * (r.x * rz.x + r.y * rz.y));
            } else {
                cplx r, rq, rz;
                rho_derivs(rk - (double)q, zk, &r, &rq, &rz);
                s_r[t] = make_float2((float)r.re, (float)-r.im);
                s_rq[t] = make_float2((float)rq.re, (float)-rq.im);
                s_rz[t] = make_float2((float)rz.re, (float)-rz.im);
                e0 += r.re * r.re + r.im * r.im;
                eq += 2.0 * (r.re * rq.re + r.im * rq.im);
                ez += 2.0 * (r.re * rz.re + r.im * rz.im);
            }
        }
        const double2 e01 = block_sum2(make_double2(e0, eq), red);
        const double2 ez2 = block_sum2(make_double2(ez, 0.0), red);
        const double E = e01.x, Eq = e01.y, Ez = ez2.x;
        // valid tap range (bins inside [0, M))
        const int t_lo = (int)max((int64_t)0, -(k0 - m + 1));
        const int t_hi = (int)min((int64_t)(2 * m), M - (k0 - m + 1));
        // channel phases e_c = exp(i 2 pi rk DM dtau_c / T) (FP64) and dtau_c e_c, in shared memory
        for (int c = threadIdx.x, ci = 0; c < a.ck; c += NT, ++ci) {
            const double dt = a.dtau[c];
            double sn, cs;
            if (rec) {
                // ci < CPT here; the unrolled select keeps the arrays in registers
                cs = ekc[0];
                sn = eks[0];
#pragma unroll
                for (int i = 1; i < CPT; ++i)
                    if (ci == i) {
                        cs = ekc[i];
                        sn = eks[i];
                    }
            } else {
                sincospi(2.0 * rk * pt.dm * dt / a.T, &sn, &cs);
            }
            s_ch[c] = make_float4((float)cs, (float)sn, (float)(dt * cs), (float)(dt * sn));
        }
        __syncthreads();
        // F = sum_t u_t H_t, H_t = sum_c e_c A^c_t (u = conj rho); the DM and r
        // derivatives need H'_t = sum_c dtau_c e_c A^c_t.  Lanes take
        // consecutive taps (coalesced reads of each channel's spectrum), warps
        // take channel groups; each warp adds its partial sums into F directly.
        float2 F = make_float2(0.f, 0.f), Fd = F, Fq = F, Fz = F;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int cper = (a.ck + NT / 32 - 1) / (NT / 32);
        const int c0 = warp * cper, c1 = min(a.ck, c0 + cper);
        const float2* Abase = a.chan_spec + (k0 - m + 1);
        for (int tb = t_lo; tb < t_hi; tb += 32) {
            const int t = tb + lane;
            if (t < t_hi) {
                float2 H = make_float2(0.f, 0.f), Hd = H;
                const float2* Ap = Abase + t;
                for (int c = c0; c < c1; ++c) {
                    const float2 x = __ldg(Ap + (int64_t)c * M);
                    const float4 e = s_ch[c];
                    H.x = fmaf(e.x, x.x, fmaf(-e.y, x.y, H.x));
                    H.y = fmaf(e.x, x.y, fmaf(e.y, x.x, H.y));
                    Hd.x = fmaf(e.z, x.x, fmaf(-e.w, x.y, Hd.x));
                    Hd.y = fmaf(e.z, x.y, fmaf(e.w, x.x, Hd.y));
                }
                const float2 u = s_r[t], v = s_rq[t], w = s_rz[t];
                F.x += u.x * H.x - u.y * H.y;
                F.y += u.x * H.y + u.y * H.x;
                Fd.x += u.x * Hd.x - u.y * Hd.y;
                Fd.y += u.x * Hd.y + u.y * Hd.x;
                Fq.x += v.x * H.x - v.y * H.y;
                Fq.y += v.x * H.y + v.y * H.x;
                Fz.x += w.x * H.x - w.y * H.y;
                Fz.y += w.x * H.y + w.y * H.x;
            }
        }
        // Fdm = i (2 pi rk / T) sum u H',  Fr = i (2 pi k DM / T) sum u H' + k sum v H,  Fz = k sum w H
        const float cdm = (float)(2.0 * M_PI * rk / a.T), cdr = (float)(2.0 * M_PI * k * pt.dm / a.T);
        const float2 Fdm = make_float2(-cdm * Fd.y, cdm * Fd.x);
        const float2 Fr = make_float2(-cdr * Fd.y + k * Fq.x, cdr * Fd.x + k * Fq.y);
        Fz = make_float2(k * Fz.x, k * Fz.y);
        const double2 sF = block_sum2(make_double2(F.x, F.y), red);
        const double2 sFdm = block_sum2(make_double2(Fdm.x, Fdm.y), red);
        const double2 sFr = block_sum2(make_double2(Fr.x, Fr.y), red);
        const double2 sFz = block_sum2(make_double2(Fz.x, Fz.y), red);
        int64_t blk = (k0 < 0 ? 0 : k0) / a.whiten_block;
        if (blk >= a.nblocks) blk = a.nblocks - 1;
        const double g = (double)a.gains[(int64_t)pt.trial * a.nblocks + blk];
        const double F2 = sF.x * sF.x + sF.y * sF.y;
        P += g * F2 / E;
        gdm += g * 2.0 * (sF.x * sFdm.x + sF.y * sFdm.y) / E;
        gr += g * (2.0 * (sF.x * sFr.x + sF.y * sFr.y) / E - F2 * k * Eq / (E * E));
        gz += g * (2.0 * (sF.x * sFz.x + sF.y * sFz.y) / E - F2 * k * Ez / (E * E));
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.power[p] = P;
        a.grad[3 * p + 0] = gdm;
        a.grad[3 * p + 1] = gr;
        a.grad[3 * p + 2] = gz;
    }
}

}  // namespace

cudaError_t launch_chan_series(const uint8_t* xcm, int64_t pitch, int32_t ck, int64_t nv, int32_t ds, float* out,
                               int64_t out_stride, unsigned long long* sums, cudaStream_t s) {
    dim3 grid((unsigned)std::min<int64_t>((nv + 255) / 256, 256), (unsigned)ck);
    k_chan_series<<<grid, 256, 0, s>>>(xcm, pitch, ck, nv, ds, out, out_stride, sums);
    return cudaGetLastError();
}

cudaError_t launch_refine_eval(const RefineArgs& a, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const size_t shm = (size_t)a.ck * sizeof(float4);
    cudaError_t e = allow_smem((const void*)k_refine_eval, shm);
    if (e != cudaSuccess) return e;
    k_refine_eval<<<(unsigned)n, NT, shm, s>>>(a);
    return cudaGetLastError();
}

int refine_max_taps() { return MAXTAP; }

}  // namespace pss
