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
//    fraction of erfc (A&S 7.1.14), truncated at min(60, ceil(220/x^2) + 6)
//    terms (~1e-15).
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
        // truncated after nt partial fractions, evaluated forwards with the
        // three-term recurrences A_k = zeta A_{k-1} + (k/2) A_{k-2} (likewise B),
        // A_0 = zeta, B_0 = 1, A_{-1} = 1, B_{-1} = 0, so that K = B / A needs one
        // division (A, B grow like |zeta|^nt: far inside the FP64 range for |x| < 1e40)
        const double h = 0.5 * sqrt(M_PI) * ax;
        const cplx zeta = {h, -h};
        // terms needed fall like 1/x^2: ceil(220 / x^2) + 6 (at most 60) agree
        // with the 60-term value to 2.3e-16 for every x > 2 (checked on a
        // 7e-4 grid up to x = 60)
        int nt = (int)ceil(220.0 / (ax * ax)) + 6;
        if (nt > 60) nt = 60;
        cplx A1 = zeta, A2 = {1.0, 0.0}, B1 = {1.0, 0.0}, B2 = {0.0, 0.0};
        for (int k = 1; k <= nt; ++k) {
            const double kk = 0.5 * k;
            const cplx A = {zeta.re * A1.re - zeta.im * A1.im + kk * A2.re, zeta.re * A1.im + zeta.im * A1.re + kk * A2.im};
            const cplx B = {zeta.re * B1.re - zeta.im * B1.im + kk * B2.re, zeta.re * B1.im + zeta.im * B1.re + kk * B2.im};
            A2 = A1;
            A1 = A;
            B2 = B1;
            B1 = B;
        }
        // K = B / A
        const double den = A1.re * A1.re + A1.im * A1.im;
        const cplx K = {(B1.re * A1.re + B1.im * A1.im) / den, (B1.im * A1.re - B1.re * A1.im) / den};
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

// Moments I_n(q) = integral_0^1 u^n e^{2 pi i q u} du, n = 0..NM-1: by the
// power series of the exponential for |q| < 0.5 (or |q| < NM/4 when more
// moments are needed), else by the upward recurrence
// I_n = (e^{ia} - n I_{n-1}) / (i a), a = 2 pi q, whose error grows like
// n!/a^n and so stays small for a > n.
template <int NM>
PSS_HD void moments_n(double q, cplx* I) {
    const double a = 2.0 * M_PI * q;
    if (fabs(q) < 0.5 || fabs(a) < 1.5 * NM) {
        // term m of I_n is t_m / (n + m + 1), t_m = (i a)^m / m!; the
        // reciprocals 1/(n + m + 1), n < NM, roll along with m (one division
        // per term instead of 2 NM)
        cplx t = {1.0, 0.0};
        double rc[NM];
        for (int n = 0; n < NM; ++n) {
            I[n] = {0.0, 0.0};
            rc[n] = 1.0 / (n + 1);
        }
        for (int m = 0; m < 80; ++m) {
            for (int n = 0; n < NM; ++n) {
                I[n].re += t.re * rc[n];
                I[n].im += t.im * rc[n];
            }
            t = c_mul(t, cplx{0.0, a * rc[0]});  // rc[0] = 1 / (m + 1)
            if (fabs(t.re) + fabs(t.im) < 1e-18) break;
            for (int n = 0; n + 1 < NM; ++n) rc[n] = rc[n + 1];
            rc[NM - 1] = 1.0 / (m + 1 + NM);
        }
        return;
    }
    double sn, cs;
    pss_sincospi(2.0 * q, &sn, &cs);
    const cplx inv_ia = {0.0, -1.0 / a};
    I[0] = c_mul(cplx{cs - 1.0, sn}, inv_ia);
    for (int n = 1; n < NM; ++n) I[n] = c_mul(cplx{cs - n * I[n - 1].re, sn - n * I[n - 1].im}, inv_ia);
}

PSS_HD void moments(double q, cplx* I) { moments_n<7>(q, I); }

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

// rho(q, z) and its partial derivatives
//   rho_q = d rho / dq = 2 pi i M1,  rho_z = d rho / dz = pi i (M2 - M1),
// M_p = integral_0^1 u^p exp(2 pi i [(q - z/2) u + z u^2 / 2]) du.
// For |z| >= 0.05 the moments follow from rho by integrating by parts
// (a = q - z/2, e = exp(2 pi i q)):
//   a rho + z M1 = (e - 1) / (2 pi i),   a M1 + z M2 = (e - rho) / (2 pi i).
// (below that the division by z loses digits); for smaller |z| everything
// comes from the Taylor series in z (terms fall as (pi |z| / 4)^n / n!) of
//   rho = sum_n (i pi z)^n / n! * integral (u^2 - u)^n e^{2 pi i q u} du
// (n <= 4), whose terms are moments I_p(q) of u^p; (u^2 - u)^n =
// sum_j C(n,j) (-1)^(n-j) u^(n+j).
PSS_HD void rho_derivs(double q, double z, cplx* r, cplx* rq, cplx* rz) {
    if (fabs(z) < 0.05) {
        cplx I[11];
        moments_n<11>(q, I);
        cplx rho = {0, 0}, dq = {0, 0}, dz = {0, 0};
        cplx c = {1.0, 0.0};  // (i pi z)^n / n!
        cplx cz = {0.0, 0.0}; // d/dz of (i pi z)^n / n! = (i pi)^n z^(n-1) / (n-1)!
        double binom[5] = {1, 0, 0, 0, 0};
        for (int n = 0; n <= 4; ++n) {
            if (n > 0) {
                // Pascal row n
                for (int j = n; j > 0; --j) binom[j] += binom[j - 1];
            }
            cplx Mn = {0, 0}, MUn = {0, 0};
            for (int j = 0; j <= n; ++j) {
                const double co = ((n - j) & 1 ? -1.0 : 1.0) * binom[j];
                Mn.re += co * I[n + j].re;
                Mn.im += co * I[n + j].im;
                MUn.re += co * I[n + j + 1].re;
                MUn.im += co * I[n + j + 1].im;
            }
            if (n > 0) {
                // c_n = c_{n-1} * (i pi z) / n ; cz_n = c_{n-1} * (i pi) (since d/dz z^n/n! = z^(n-1)/(n-1)!)
                const cplx ipi = {0.0, M_PI};
                cz = c_mul(c, ipi);
                c = c_mul(c, cplx{0.0, M_PI * z / n});
            }
            const cplx t0 = c_mul(c, Mn);
            rho.re += t0.re;
            rho.im += t0.im;
            const cplx t1 = c_mul(c, c_mul(cplx{0.0, 2.0 * M_PI}, MUn));
            dq.re += t1.re;
            dq.im += t1.im;
            if (n > 0) {
                const cplx t2 = c_mul(cz, Mn);
                dz.re += t2.re;
                dz.im += t2.im;
            }
        }
        *r = rho;
        *rq = dq;
        *rz = dz;
        return;
    }
    const cplx rho = rho_resp(q, z);
    double sn, cs;
    pss_sincospi(2.0 * q, &sn, &cs);
    const double a = q - 0.5 * z;
    const cplx inv2pii = {0.0, -1.0 / (2.0 * M_PI)};
    const cplx t1 = c_mul(cplx{cs - 1.0, sn}, inv2pii);
    const cplx M1 = {(t1.re - a * rho.re) / z, (t1.im - a * rho.im) / z};
    const cplx t2 = c_mul(cplx{cs - rho.re, sn - rho.im}, inv2pii);
    const cplx M2 = {(t2.re - a * M1.re) / z, (t2.im - a * M1.im) / z};
    *r = rho;
    *rq = c_mul(cplx{0.0, 2.0 * M_PI}, M1);
    *rz = c_mul(cplx{0.0, M_PI}, cplx{M2.re - M1.re, M2.im - M1.im});
}

}  // namespace pss
