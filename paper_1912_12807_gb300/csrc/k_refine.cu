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
// Phases and the response (rho_derivs, response.cuh) are evaluated in FP64
// (harmonic k's channel phases as the k-th power of the fundamental's);
// the channel sums accumulate in FP32 and are reduced across the CTA in FP64.
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
            cplx r, rq, rz;
            rho_derivs(rk - (double)q, zk, &r, &rq, &rz);
            s_r[t] = make_float2((float)r.re, (float)-r.im);
            s_rq[t] = make_float2((float)rq.re, (float)-rq.im);
            s_rz[t] = make_float2((float)rz.re, (float)-rz.im);
            e0 += r.re * r.re + r.im * r.im;
            eq += 2.0 * (r.re * rq.re + r.im * rq.im);
            ez += 2.0 * (r.re * rz.re + r.im * rz.im);
        }
        const double2 e01 = block_sum2(make_double2(e0, eq), red);
        const double2 ez2 = block_sum2(make_double2(ez, 0.0), red);
        const double E = e01.x, Eq = e01.y, Ez = ez2.x;
        // valid tap range (bins inside [0, M))
        const int t_lo = (int)max((int64_t)0, -(k0 - m + 1));
        const int t_hi = (int)min((int64_t)(2 * m), M - (k0 - m + 1));
        float2 F = make_float2(0.f, 0.f), Fdm = F, Fr = F, Fz = F;
        for (int c = threadIdx.x, ci = 0; c < a.ck; c += NT, ++ci) {
            const float2* Ac = a.chan_spec + (int64_t)c * M + (k0 - m + 1);
            float2 G = make_float2(0.f, 0.f), Gq = G, Gz = G;
            for (int t = t_lo; t < t_hi; ++t) {
                const float2 x = __ldg(Ac + t);
                const float2 u = s_r[t], v = s_rq[t], w = s_rz[t];
                G.x = fmaf(x.x, u.x, fmaf(-x.y, u.y, G.x));
                G.y = fmaf(x.x, u.y, fmaf(x.y, u.x, G.y));
                Gq.x = fmaf(x.x, v.x, fmaf(-x.y, v.y, Gq.x));
                Gq.y = fmaf(x.x, v.y, fmaf(x.y, v.x, Gq.y));
                Gz.x = fmaf(x.x, w.x, fmaf(-x.y, w.y, Gz.x));
                Gz.y = fmaf(x.x, w.y, fmaf(x.y, w.x, Gz.y));
            }
            // phase exp(i 2 pi rk DM dtau_c / T), FP64
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
            const float2 e = make_float2((float)cs, (float)sn);
            const float2 eG = make_float2(e.x * G.x - e.y * G.y, e.x * G.y + e.y * G.x);
            F.x += eG.x;
            F.y += eG.y;
            // i * dphi * eG
            const float dphi_dm = (float)(2.0 * M_PI * rk * dt / a.T);
            const float dphi_dr = (float)(2.0 * M_PI * k * pt.dm * dt / a.T);
            Fdm.x += -dphi_dm * eG.y;
            Fdm.y += dphi_dm * eG.x;
            const float2 eGq = make_float2(e.x * Gq.x - e.y * Gq.y, e.x * Gq.y + e.y * Gq.x);
            Fr.x += -dphi_dr * eG.y + k * eGq.x;
            Fr.y += dphi_dr * eG.x + k * eGq.y;
            const float2 eGz = make_float2(e.x * Gz.x - e.y * Gz.y, e.x * Gz.y + e.y * Gz.x);
            Fz.x += k * eGz.x;
            Fz.y += k * eGz.y;
        }
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
    k_refine_eval<<<(unsigned)n, NT, 0, s>>>(a);
    return cudaGetLastError();
}

int refine_max_taps() { return MAXTAP; }

}  // namespace pss
