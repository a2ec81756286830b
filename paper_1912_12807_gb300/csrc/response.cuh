// Response of a linearly drifting sinusoid, FP64, device and host.
//
//   rho(q, z) = integral_0^1 exp(2 pi i [(q - z/2) u + z u^2 / 2]) du
//
// is the DFT at bin k (q = r - k) of a unit signal whose frequency moves from
// r - z/2 to r + z/2 bins over the series (the template behind the paper's
// accelsearch zmax, Sect. 3.2).  Evaluation:
//  * z == 0: exp(i pi q) sin(pi q) / (pi q) (sinpi/cospi: exact zeros at
//    integer q != 0).
//  * 0 < |z| < 1e-2: third-order Taylor expansion in z, using the moments
//    I_n(q) = integral_0^1 u^n exp(2 pi i q u) du (n <= 6).
//  * otherwise: completing the square gives Fresnel integrals,
//      rho = exp(-i pi (q - z/2)^2 / z) [dC + i sgn(z) dS] / sqrt(2|z|),
//      dC = C(w1) - C(w0), w0 = sqrt(2|z|) b, w1 = sqrt(2|z|) (1 + b),
//      b = (q - z/2) / z,
//    with C + iS = ((1+i)/2) erf(sqrt(pi) (1-i) x / 2) (Abramowitz & Stegun
//    7.3.22) evaluated by the power series (A&S 7.3.11, 7.3.13) for |x| <= 2
//    and, above, by the auxiliary functions f, g through the continued
//    fraction of erfc (A&S 7.1.14), truncated at 60 terms (~1e-15).
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define PSS_HD __host__ __device__ __forceinline__
#else
#define PSS_HD inline
#endif

namespace pss {

struct cplx {
    double re, im;
};

PSS_HD cplx c_mul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

PSS_HD void pss_sincospi(double x, double* s, double* c) {
#ifdef __CUDA_ARCH__
    sincospi(x, s, c);
#else
    // reduce x modulo 2 exactly, then call the libm routines on pi*r
    double r = fmod(x, 2.0);
    if (r < -1.0) r += 2.0;
    if (r > 1.0) r -= 2.0;
    *s = sin(M_PI * r);
    *c = cos(M_PI * r);
    if (r == 0.0 || r == 1.0 || r == -1.0) *s = 0.0;
    if (r == 0.5 || r == -0.5) *c = 0.0;
#endif
}

// Fresnel integrals C(x), S(x) with kernels cos / sin (pi t^2 / 2).
PSS_HD void fresnel_cs(double x, double* C, double* S) {
    const double ax = fabs(x);
    double c, s;
    if (ax <= 2.0) {
        // term_k = (pi/2)^k x^(2k+1) / k!, divided by (2k+1); signs and targets
        // cycle C+, S+, C-, S-.
        double t = ax;
        c = 0.0;
        s = 0.0;
        const double a2 = 0.5 * M_PI * ax * ax;
        for (int k = 0; k < 60; ++k) {
            const double term = t / (2 * k + 1);
            switch (k & 3) {
                case 0: c += term; break;
                case 1: s += term; break;
                case 2: c -= term; break;
                default: s -= term; break;
            }
            t *= a2 / (k + 1);
            if (t < 1e-18) break;
        }
    } else {
        // zeta = sqrt(pi) (1 - i) x / 2;  K = 1 / (zeta + (1/2)/(zeta + (2/2)/(zeta + ...)))
        const double h = 0.5 * sqrt(M_PI) * ax;
        cplx zeta = {h, -h};
        cplx cf = zeta;
        for (int k = 60; k >= 1; --k) {
            // cf = zeta + (k/2) / cf
            const double den = cf.re * cf.re + cf.im * cf.im;
            const double kk = 0.5 * k;
            cf = {zeta.re + kk * cf.re / den, zeta.im - kk * cf.im / den};
        }
        const double den = cf.re * cf.re + cf.im * cf.im;
        const cplx K = {cf.re / den, -cf.im / den};
        // g + i f = (1 + i) / (2 sqrt(pi)) * K
        const double fac = 0.5 / sqrt(M_PI);
        const double g = fac * (K.re - K.im);
        const double f = fac * (K.re + K.im);
        double sn, cs;
        pss_sincospi(0.5 * ax * ax, &sn, &cs);
        c = 0.5 + f * sn - g * cs;
        s = 0.5 - f * cs - g * sn;
    }
    if (x < 0) {
        c = -c;
        s = -s;
    }
    *C = c;
    *S = s;
}

// Moments I_n(q) = integral_0^1 u^n e^{2 pi i q u} du, n = 0..6: by the
// power series of the exponential for |q| < 0.5, else by the upward
// recurrence I_n = (e^{ia} - n I_{n-1}) / (i a), a = 2 pi q (stable there).
PSS_HD void moments(double q, cplx* I) {
    const double a = 2.0 * M_PI * q;
    if (fabs(q) < 0.5) {
        cplx t = {1.0, 0.0};
        for (int n = 0; n <= 6; ++n) I[n] = {0.0, 0.0};
        for (int m = 0; m < 40; ++m) {
            for (int n = 0; n <= 6; ++n) {
                I[n].re += t.re / (n + m + 1);
                I[n].im += t.im / (n + m + 1);
            }
            t = c_mul(t, cplx{0.0, a / (m + 1)});
        }
        return;
    }
    double sn, cs;
    pss_sincospi(2.0 * q, &sn, &cs);
    const cplx inv_ia = {0.0, -1.0 / a};
    I[0] = c_mul(cplx{cs - 1.0, sn}, inv_ia);
    for (int n = 1; n <= 6; ++n) I[n] = c_mul(cplx{cs - n * I[n - 1].re, sn - n * I[n - 1].im}, inv_ia);
}

PSS_HD cplx rho_resp(double q, double z) {
    if (z == 0.0) {
        double sn, cs;
        pss_sincospi(q, &sn, &cs);
        if (q == 0.0) return {1.0, 0.0};
        const double sc = sn / (M_PI * q);
        return {cs * sc, sn * sc};
    }
    if (fabs(z) < 1e-2) {
        // rho = sum_n (i pi z)^n / n! * integral (u^2 - u)^n e^{2 pi i q u} du,
        // |u^2 - u| <= 1/4, so the terms fall as (pi |z| / 4)^n / n!: n <= 3
        // leaves < 2e-10 for |z| < 1e-2.
        cplx I[7];
        moments(q, I);
        cplx M[4];
        M[0] = I[0];
        M[1] = {I[2].re - I[1].re, I[2].im - I[1].im};
        M[2] = {I[4].re - 2 * I[3].re + I[2].re, I[4].im - 2 * I[3].im + I[2].im};
        M[3] = {I[6].re - 3 * I[5].re + 3 * I[4].re - I[3].re, I[6].im - 3 * I[5].im + 3 * I[4].im - I[3].im};
        cplx acc = M[0];
        cplx f = {1.0, 0.0};
        for (int n = 1; n <= 3; ++n) {
            f = c_mul(f, cplx{0.0, M_PI * z / n});
            const cplx t = c_mul(f, M[n]);
            acc.re += t.re;
            acc.im += t.im;
        }
        return acc;
    }
    const double az = fabs(z);
    const double sq = sqrt(2.0 * az);
    const double bb = (q - 0.5 * z) / z;
    double C0, S0, C1, S1;
    fresnel_cs(sq * bb, &C0, &S0);
    fresnel_cs(sq * (1.0 + bb), &C1, &S1);
    const double dC = (C1 - C0) / sq;
    const double dS = (z > 0 ? 1.0 : -1.0) * (S1 - S0) / sq;
    const double qq = q - 0.5 * z;
    double sn, cs;
    pss_sincospi(-(qq * qq) / z, &sn, &cs);
    return c_mul(cplx{cs, sn}, cplx{dC, dS});
}

}  // namespace pss
