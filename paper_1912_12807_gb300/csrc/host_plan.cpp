// Dedispersion plan (DDplan; paper Sect. 3.1, Tables 2-3) and detection
// statistics, host side.  Compiled with -ffp-contract=off so the FP64
// expressions below are evaluated exactly in the order written.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>
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

// N_v and nfft of every stage from the plan's largest delay.
static pss_status set_lengths(Plan* P) {
    if (P->nsamp <= P->max_delay) return fail(PSS_EINVAL, "pss_dd_plan: file shorter than the largest dispersion delay");
    for (auto& si : P->stages) {
        si.nv = (P->nsamp - P->max_delay) / si.ds;
        if (si.nv < 1) return fail(PSS_EINVAL, "pss_dd_plan: no valid samples after downsampling");
        si.nfft = next_pow2(si.nv);
        if (si.nfft > (int64_t(1) << 24)) return fail(PSS_EINVAL, "pss_dd_plan: series longer than 2^24");
    }
    return PSS_OK;
}

pss_status build_plan(const pss_fil_desc* fil, const pss_dd_stage* st, int nst, Plan* P) {
    static std::atomic<uint64_t> next_id{1};
    P->id = next_id.fetch_add(1);
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
    P->nsub = 0;
    return set_lengths(P);
}

// Two-stage (prepsubband) scheme; the paper only says it is faster than one
// prepdata per DM (Sect. 5).  Subband b = channels [b S, (b+1) S), reference
// f_b = its highest centre frequency; groups of `group` consecutive trials
// of one stage, nominal DM = the middle trial's (index first + (n-1)/2);
//   e_c(g)  = round(((K DM_g) (1/(f_c f_c) - 1/(f_b f_b))) / tsamp),
//   D_b(i)  = round(((K DM_i) (1/(f_b f_b) - 1/(f_ref f_ref))) / tsamp),
// halves away from zero; D' = max(D, max_{i,c} e_c(g_i) + D_b(c)(i)).
pss_status build_subband(Plan* P, int32_t nsub, int32_t group) {
    const int C = P->nchan;
    if (nsub < 1 || C % nsub != 0) return fail(PSS_EINVAL, "pss_dd_plan_subband: nsub must divide nchan");
    if (group < 1 || group > 1024) return fail(PSS_EINVAL, "pss_dd_plan_subband: group must be in [1, 1024]");
    const int S = C / nsub;
    P->nsub = nsub;
    P->sub_group = group;
    P->sub_S = S;
    double fref = -1e300;
    for (int c = 0; c < C; ++c) fref = std::max(fref, P->freqs[c]);
    P->fsub.assign(nsub, -1e300);
    for (int c = 0; c < C; ++c) P->fsub[c / S] = std::max(P->fsub[c / S], P->freqs[c]);
    const int64_t ndm = P->ndm();
    P->grp_first.clear();
    P->grp_n.clear();
    P->grp_dm.clear();
    P->grp_of.assign(ndm, 0);
    for (int64_t i = 0; i < ndm;) {
        int64_t j = i;
        while (j < ndm && j - i < group && P->stage_of[j] == P->stage_of[i]) ++j;
        for (int64_t k = i; k < j; ++k) P->grp_of[k] = (int32_t)P->grp_first.size();
        P->grp_first.push_back(i);
        P->grp_n.push_back((int32_t)(j - i));
        P->grp_dm.push_back(P->dms[i + (j - i - 1) / 2]);
        i = j;
    }
    const int64_t ng = (int64_t)P->grp_first.size();
    P->sub_e.assign((size_t)ng * C, 0);
    P->sub_D.assign((size_t)ndm * nsub, 0);
    std::vector<double> din(C), db(nsub);
    for (int c = 0; c < C; ++c) {
        const double fb = P->fsub[c / S];
        din[c] = 1.0 / (P->freqs[c] * P->freqs[c]) - 1.0 / (fb * fb);
    }
    for (int b = 0; b < nsub; ++b) db[b] = 1.0 / (P->fsub[b] * P->fsub[b]) - 1.0 / (fref * fref);
    for (int64_t g = 0; g < ng; ++g) {
        const double kd = K_DISP * P->grp_dm[g];
        for (int c = 0; c < C; ++c) {
            const double r = round((kd * din[c]) / P->tsamp);
            if (!(r < 2.0e9)) return fail(PSS_EINVAL, "pss_dd_plan_subband: delay exceeds int32");
            P->sub_e[(size_t)g * C + c] = (int32_t)r;
        }
    }
    int64_t dmax = P->max_delay;
    for (int64_t i = 0; i < ndm; ++i) {
        const double kd = K_DISP * P->dms[i];
        for (int b = 0; b < nsub; ++b) {
            const double r = round((kd * db[b]) / P->tsamp);
            if (!(r < 2.0e9)) return fail(PSS_EINVAL, "pss_dd_plan_subband: delay exceeds int32");
            P->sub_D[(size_t)i * nsub + b] = (int32_t)r;
        }
        const int32_t* e = &P->sub_e[(size_t)P->grp_of[i] * C];
        for (int c = 0; c < C; ++c) dmax = std::max<int64_t>(dmax, (int64_t)e[c] + P->sub_D[(size_t)i * nsub + c / S]);
    }
    P->max_delay = dmax;
    return set_lengths(P);
}

// ---- automatic plan (DDplan-like; the paper's Tables 2-3 come from DDplan.py,
// Sect. 3.1) ------------------------------------------------------------------
// Smearing terms (nu = band centre in GHz, widths in MHz, seconds):
//   t_chan(DM) = 8.3e-6 DM dnu / nu^3,   t_bw(d) = 8.3e-6 d BW / nu^3.
// Nominal factor v starts at the smallest power of two with v tsamp >= tres
// (capped at ds_max) and doubles per stage; a stage downsamples by
// min(v, ds_max), takes the largest listed step s with t_bw(s/2) <=
// sqrt(ts^2 + t_chan(d0)^2), and runs to where t_chan reaches kappa v tsamp
// (at least one step, at most dm_hi), kappa = 3.5.
pss_status auto_plan(const pss_fil_desc* fil, double dm_lo, double dm_hi, double tres, int32_t ds_max,
                     std::vector<pss_dd_stage>* rows) {
    static const double kSteps[] = {0.01, 0.02, 0.03, 0.05, 0.1, 0.2, 0.3, 0.5, 1.0, 2.0, 3.0, 5.0, 10.0,
                                    20.0, 30.0, 50.0, 100.0, 200.0, 300.0, 500.0, 1000.0};
    const double kappa = 3.5;
    const int nchan = fil->nchan;
    const double ctr = fil->fch0_mhz + 0.5 * (double)(nchan - 1) * fil->foff_mhz;
    const double dnu = fabs(fil->foff_mhz), bw = (double)nchan * fabs(fil->foff_mhz);
    const double nu = ctr / 1000.0;
    const double kch = 8.3e-6 * dnu / (nu * nu * nu);
    const double kbw = 8.3e-6 * bw / (nu * nu * nu);
    int64_t v = 1;
    while (v < ds_max && (double)v * fil->tsamp_s < tres) v *= 2;
    double d0 = dm_lo;
    rows->clear();
    while (d0 < dm_hi) {
        if (rows->size() > 4096) return fail(PSS_EINVAL, "pss_dd_plan_auto: more than 4096 rows");
        const int64_t ds = std::min<int64_t>(v, ds_max);
        const double ts = (double)ds * fil->tsamp_s;
        const double tc = kch * d0;
        const double T = sqrt(ts * ts + tc * tc);
        double step = kSteps[0];
        for (double st : kSteps)
            if (kbw * (0.5 * st) <= T) step = st;
        const double dsw = kappa * ((double)v * fil->tsamp_s) / kch;
        const double end = std::min(std::max(dsw, d0 + step), dm_hi);
        int64_t n = (int64_t)ceil((end - d0) / step - 1e-9);
        if (n < 1) n = 1;
        if (n > (int64_t)1 << 30) return fail(PSS_EINVAL, "pss_dd_plan_auto: too many trials in a row");
        pss_dd_stage r;
        r.dm_lo = d0;
        r.dm_step = step;
        r.n_dm = (int32_t)n;
        r.ds = (int32_t)ds;
        rows->push_back(r);
        d0 = d0 + (double)n * step;
        if (v < ((int64_t)1 << 40)) v *= 2;
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

extern "C" pss_status pss_dd_plan_auto(const pss_fil_desc* fil, double dm_lo, double dm_hi, double tres_s,
                                       int32_t ds_max, pss_dd_stage* out, int32_t cap, int32_t* n_out) {
    if (!fil || !n_out) return pss::fail(PSS_EINVAL, "pss_dd_plan_auto: null argument");
    *n_out = 0;
    if (fil->nchan <= 0 || !(fil->tsamp_s > 0) || !(fil->foff_mhz != 0))
        return pss::fail(PSS_EINVAL, "pss_dd_plan_auto: bad descriptor");
    if (!(dm_lo >= 0) || !(dm_hi > dm_lo) || !std::isfinite(dm_hi) || !std::isfinite(tres_s))
        return pss::fail(PSS_EINVAL, "pss_dd_plan_auto: need 0 <= dm_lo < dm_hi, finite");
    if (ds_max < 1 || ds_max > 1024 || (ds_max & (ds_max - 1)))
        return pss::fail(PSS_EINVAL, "pss_dd_plan_auto: ds_max must be a power of two in [1, 1024]");
    const double ctr = fil->fch0_mhz + 0.5 * (double)(fil->nchan - 1) * fil->foff_mhz;
    if (!(ctr > 0)) return pss::fail(PSS_EINVAL, "pss_dd_plan_auto: band centre must be > 0");
    std::vector<pss_dd_stage> rows;
    pss_status st = pss::auto_plan(fil, dm_lo, dm_hi, tres_s, ds_max, &rows);
    if (st != PSS_OK) return st;
    *n_out = (int32_t)rows.size();
    if ((int32_t)rows.size() > cap) return pss::fail(PSS_ECAP, "pss_dd_plan_auto: more rows than cap");
    if (!rows.empty()) memcpy(out, rows.data(), rows.size() * sizeof(pss_dd_stage));
    return PSS_OK;
}

extern "C" double pss_sigma_of_power(int32_t numharm, double power) {
    if (numharm < 1) return 0.0;
    return pss::sigma_of_power(numharm, power);
}
extern "C" double pss_power_threshold(int32_t numharm, double sigma) {
    if (numharm < 1) return 0.0;
    return pss::power_threshold(numharm, sigma);
}
