// Dedispersion plan (DDplan; paper Sect. 3.1, Tables 2-3) and detection
// statistics, host side.  Compiled with -ffp-contract=off so the FP64
// expressions below are evaluated exactly in the order written.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "pss_internal.h"

namespace pss {

thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
pss_status fail(pss_status st, const std::string& msg) {
    g_err = msg;
    return st;
}
pss_status cuda_fail(cudaError_t e, const char* what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return PSS_ECUDA;
}

static const double K_DISP = 4.148808e3;  // s MHz^2 pc^-1 cm^3

static int64_t next_pow2(int64_t n) {
    int64_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

pss_status build_plan(const pss_fil_desc* fil, const pss_dd_stage* st, int nst, Plan* P) {
    if (!fil || !st || nst <= 0) return fail(PSS_EINVAL, "pss_dd_plan: null descriptor or no stages");
    if (fil->nchan <= 0 || fil->nsamp <= 0) return fail(PSS_EINVAL, "pss_dd_plan: nchan and nsamp must be > 0");
    if (!(fil->tsamp_s > 0)) return fail(PSS_EINVAL, "pss_dd_plan: tsamp_s must be > 0");
    if (fil->nbits != 8 && fil->nbits != 1) return fail(PSS_EINVAL, "pss_dd_plan: nbits must be 8 or 1");
    P->nchan = fil->nchan;
    P->nsamp = fil->nsamp;
    P->tsamp = fil->tsamp_s;
    P->fch0 = fil->fch0_mhz;
    P->foff = fil->foff_mhz;
    P->freqs.resize(fil->nchan);
    double fmax = -1e300;
    for (int c = 0; c < fil->nchan; ++c) {
        // f_c = fch0 + c*foff: channel 0's centre plus c spacings.
        P->freqs[c] = fil->fch0_mhz + (double)c * fil->foff_mhz;
        if (!(P->freqs[c] > 0)) return fail(PSS_EINVAL, "pss_dd_plan: channel frequencies must be > 0");
        fmax = std::max(fmax, P->freqs[c]);
    }
    P->stages.clear();
    P->dms.clear();
    P->stage_of.clear();
    int64_t first = 0;
    for (int s = 0; s < nst; ++s) {
        if (st[s].n_dm <= 0) return fail(PSS_EINVAL, "pss_dd_plan: stage with n_dm <= 0");
        int ds = st[s].ds;
        if (ds < 1 || ds > 1024 || (ds & (ds - 1)) != 0)
            return fail(PSS_EINVAL, "pss_dd_plan: ds must be a power of two in [1, 1024]");
        StageInfo si;
        si.dm_lo = st[s].dm_lo;
        si.dm_step = st[s].dm_step;
        si.n_dm = st[s].n_dm;
        si.ds = ds;
        si.first = first;
        for (int i = 0; i < st[s].n_dm; ++i) {
            // DM_i = lo + i*step, each value computed directly.
            double dm = st[s].dm_lo + (double)i * st[s].dm_step;
            if (dm < 0) return fail(PSS_EINVAL, "pss_dd_plan: negative DM");
            P->dms.push_back(dm);
            P->stage_of.push_back(s);
        }
        first += st[s].n_dm;
        P->stages.push_back(si);
    }
    const int64_t ndm = (int64_t)P->dms.size();
    const int C = fil->nchan;
    P->delays.assign((size_t)ndm * C, 0);
    const double inv_ref = 1.0 / (fmax * fmax);
    std::vector<double> diff(C);
    for (int c = 0; c < C; ++c) diff[c] = 1.0 / (P->freqs[c] * P->freqs[c]) - inv_ref;
    int64_t dmax = 0;
    for (int64_t i = 0; i < ndm; ++i) {
        const double kd = K_DISP * P->dms[i];
        for (int c = 0; c < C; ++c) {
            double v = (kd * diff[c]) / fil->tsamp_s;
            double r = round(v);  // halves away from zero
            if (!(r < 2.0e9)) return fail(PSS_EINVAL, "pss_dd_plan: delay exceeds int32");
            P->delays[(size_t)i * C + c] = (int32_t)r;
            dmax = std::max<int64_t>(dmax, (int64_t)r);
        }
    }
    P->max_delay = dmax;
    if (fil->nsamp <= dmax) return fail(PSS_EINVAL, "pss_dd_plan: file shorter than the largest dispersion delay");
    for (auto& si : P->stages) {
        si.nv = (fil->nsamp - dmax) / si.ds;
        if (si.nv < 1) return fail(PSS_EINVAL, "pss_dd_plan: no valid samples after downsampling");
        si.nfft = next_pow2(si.nv);
        if (si.nfft > (int64_t(1) << 24)) return fail(PSS_EINVAL, "pss_dd_plan: series longer than 2^24");
    }
    return PSS_OK;
}

// ---- statistics -----------------------------------------------------------
// Noise powers are Exp(1); a sum of n of them is Gamma(n, 1) with tail
// Q(n, S) = exp(-S) sum_{j<n} S^j / j!.  sigma = -Phi^-1(Q).

namespace {
// lgamma(j + 1) for j < 64
struct LogFactorials {
    double v[64];
    LogFactorials() {
        for (int j = 0; j < 64; ++j) v[j] = lgamma((double)j + 1.0);
    }
};
const LogFactorials kLogFact;
}  // namespace

double log_q(int n, double S) {
    if (S <= 0) return 0.0;
    if (n > 64) n = 64;
    const double lS = log(S);
    if (S >= n) {
        // The terms grow with j up to j = n - 1; relative to the last one,
        // term_j / term_{n-1} = prod_{i=j+1}^{n-1} i / S <= 1.
        double ratio = 1.0, acc = 1.0;
        for (int j = n - 2; j >= 0; --j) {
            ratio *= (double)(j + 1) / S;
            acc += ratio;
        }
        return (n - 1) * lS - S - kLogFact.v[n - 1] + log(acc);
    }
    double mx = -1e300;
    double t[64];
    for (int j = 0; j < n; ++j) {
        t[j] = j * lS - S - kLogFact.v[j];
        mx = std::max(mx, t[j]);
    }
    double acc = 0;
    for (int j = 0; j < n; ++j) acc += exp(t[j] - mx);
    return mx + log(acc);
}

// log Phi(-x) for x >= 0: from erfc while it does not underflow, then the
// asymptotic (Laplace) continued-fraction form of the Mills ratio.
static double log_phi_neg(double x) {
    if (x < 25.0) return log(0.5 * erfc(x / sqrt(2.0)));
    // Mills ratio R(x) = Phi(-x)/phi(x) by its continued fraction
    // R = 1/(x + 1/(x + 2/(x + 3/(x + ...)))), evaluated bottom-up.
    double cf = x;
    for (int k = 60; k >= 1; --k) cf = x + k / cf;
    double R = 1.0 / cf;
    return -0.5 * x * x - 0.5 * log(2.0 * M_PI) + log(R);
}

double sigma_from_logp(double logp) {
    if (logp >= log(0.5)) {
        // p >= 0.5: sigma <= 0; solve on the other branch by symmetry.
        double q = -expm1(logp);  // 1 - p without cancellation; sigma = -sigma_from(q)
        if (q <= 0) return -40.0;
        return -sigma_from_logp(log(q));
    }
    // Newton on g(x) = log Phi(-x) - logp, g'(x) = -phi(x)/Phi(-x).
    double t = -2.0 * logp;
    double x = sqrt(std::max(t - log(std::max(t, 1.0) * 2.0 * M_PI), 0.01));
    for (int it = 0; it < 100; ++it) {
        double lp = log_phi_neg(x);
        double lphi = -0.5 * x * x - 0.5 * log(2.0 * M_PI);
        double dg = -exp(lphi - lp);
        double step = (lp - logp) / dg;
        x -= step;
        if (x < 0) x = 0;
        if (fabs(step) < 1e-14 * std::max(1.0, x)) break;
    }
    return x;
}

double sigma_of_power(int n, double S) { return sigma_from_logp(log_q(n, S)); }

double power_threshold(int n, double sigma) {
    double lo = 0.0, hi = 10.0;
    while (sigma_of_power(n, hi) < sigma) hi *= 2.0;
    for (int i = 0; i < 200; ++i) {
        double mid = 0.5 * (lo + hi);
        if (sigma_of_power(n, mid) < sigma) lo = mid;
        else hi = mid;
        if (hi - lo <= 1e-13 * hi) break;
    }
    return hi;
}

}  // namespace pss

extern "C" const char* pss_last_error(void) { return pss::g_err.c_str(); }

extern "C" double pss_sigma_of_power(int32_t numharm, double power) {
    if (numharm < 1) return 0.0;
    return pss::sigma_of_power(numharm, power);
}
extern "C" double pss_power_threshold(int32_t numharm, double sigma) {
    if (numharm < 1) return 0.0;
    return pss::power_threshold(numharm, sigma);
}
