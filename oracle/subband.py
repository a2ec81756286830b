"""Two-stage (subband) dedispersion, the prepsubband scheme.

TEST INFRASTRUCTURE: like the rest of `oracle/`, only the tests, the smoke
check and the CPU-baseline leg of the benchmark use this module.

The paper runs one prepdata process per DM and remarks that prepsubband,
which shares partial sums between DMs, is faster (Sect. 5, "Using other
routines").  It gives no formulas; this is the reading used here:

* Subbands.  nsub subbands of S = nchan / nsub consecutive channels.
  Subband b's reference frequency f_b is the highest centre frequency among
  its channels.
* Groups.  The trials of each plan stage are cut into groups of `group`
  consecutive trials (the last group of a stage may be shorter).  Group g's
  nominal DM is the DM of its middle trial, index first + (n_g - 1) // 2.
* Stage 1, per group g and subband b:
      u_{g,b}[t] = sum over kept channels c of b of x[c][t + e_c(g)],
      e_c(g) = round_half_away(((K * DM_g) * (1/(f_c f_c) - 1/(f_b f_b))) / tsamp).
* Stage 2, per trial i of group g:
      s_i[t] = sum_b u_{g,b}[t + D_b(i)],
      D_b(i) = round_half_away(((K * DM_i) * (1/(f_b f_b) - 1/(f_ref f_ref))) / tsamp),
  for t < N - D', then the boxcar of ds samples as in the exact scheme.
  f_ref is the highest channel frequency of the file.
* D' = max(D, max over trials i and channels c of e_c(g_i) + D_{b(c)}(i)),
  D the exact plan's largest delay, so that every read stays inside the
  file; the stage lengths follow from D' as the exact plan's follow from D.

e_c(g) + D_b(i) approximates the exact delay d_c(i): the two differ by the
channel's within-subband delay at DM_i - DM_g plus at most three roundings:
the smearing the scheme trades for its shared partial sums.  With S = 1
(nsub = nchan), or with nsub = 1 and groups of one trial, the scheme is the
exact one.
Every FP64 expression is evaluated in the order written.
"""
from __future__ import annotations

import numpy as np

from . import plan as _plan


class SubbandPlan:
    """Tables of the two-stage scheme for a DM grid (see module docstring).

    Attributes: nsub, group, S; fsub [nsub] (f_b); grp_first, grp_n,
    grp_dm [ngroups]; grp_of [ndm]; e [ngroups][nchan] (int64, e_c(g));
    D [ndm][nsub] (int64, D_b(i)); max_comb (largest e + D)."""

    def __init__(self, freqs, dms, stage_of, tsamp_s, nsub: int, group: int):
        freqs = np.asarray(freqs, dtype=np.float64)
        nchan = freqs.shape[0]
        if nsub < 1 or nchan % nsub != 0:
            raise ValueError("nsub must divide nchan")
        if group < 1:
            raise ValueError("group must be >= 1")
        self.nsub, self.group, self.S = int(nsub), int(group), nchan // int(nsub)
        S = self.S
        self.fsub = np.array([freqs[b * S:(b + 1) * S].max() for b in range(nsub)])
        f_ref = float(freqs.max())
        dms = np.asarray(dms, dtype=np.float64)
        stage_of = np.asarray(stage_of)
        # groups: consecutive trials of one stage
        first, n, gdm, grp_of = [], [], [], np.empty(len(dms), dtype=np.int64)
        i = 0
        while i < len(dms):
            j = i
            while j < len(dms) and j - i < group and stage_of[j] == stage_of[i]:
                j += 1
            grp_of[i:j] = len(first)
            first.append(i)
            n.append(j - i)
            gdm.append(float(dms[i + (j - i - 1) // 2]))
            i = j
        self.grp_first = np.array(first, dtype=np.int64)
        self.grp_n = np.array(n, dtype=np.int64)
        self.grp_dm = np.array(gdm, dtype=np.float64)
        self.grp_of = grp_of
        # within-subband delays at the nominal DM
        fb_c = np.repeat(self.fsub, S)
        diff_in = 1.0 / (freqs * freqs) - 1.0 / (fb_c * fb_c)
        kd = _plan.K_DM * self.grp_dm
        self.e = _plan.round_half_away((kd[:, None] * diff_in[None, :]) / tsamp_s)
        # subband delays at each trial's DM
        diff_b = 1.0 / (self.fsub * self.fsub) - 1.0 / (f_ref * f_ref)
        kd = _plan.K_DM * dms
        self.D = _plan.round_half_away((kd[:, None] * diff_b[None, :]) / tsamp_s)
        comb = self.e[self.grp_of] + np.repeat(self.D, S, axis=1) if len(dms) else np.zeros((0, nchan))
        self.max_comb = int(comb.max()) if comb.size else 0

    def combined_delays(self, dm_idx: int) -> np.ndarray:
        """e_c(g_i) + D_{b(c)}(i) for every channel of trial dm_idx."""
        return self.e[self.grp_of[dm_idx]] + np.repeat(self.D[dm_idx], self.S)


def stage1(x_cm: np.ndarray, sp: SubbandPlan, g: int, lengths, chan_mask=None):
    """u_{g,b}[t] for t < lengths[b], one int64 array per subband b."""
    nchan = x_cm.shape[0]
    u = [np.zeros(int(n), dtype=np.int64) for n in lengths]
    for c in range(nchan):
        if chan_mask is not None and not chan_mask[c]:
            continue
        e, b = int(sp.e[g, c]), c // sp.S
        u[b] += x_cm[c, e:e + int(lengths[b])].astype(np.int64)
    return u


def dedisperse_subband(x_cm: np.ndarray, sp: SubbandPlan, dm_idx: int, max_delay: int, ds: int,
                       chan_mask=None) -> np.ndarray:
    """int64 [N_v] of trial dm_idx by the two stages (module docstring);
    max_delay is the plan's D'.  Stage 1 is evaluated over the samples this
    trial reads, t < N - D' + D_b(i) (which stays inside the file because
    e_c + D_b(i) <= D')."""
    nsamp = x_cm.shape[1]
    L = nsamp - int(max_delay)
    Dm = sp.D[dm_idx]
    u = stage1(x_cm, sp, int(sp.grp_of[dm_idx]), [L + int(d) for d in Dm], chan_mask)
    s = np.zeros(L, dtype=np.int64)
    for b in range(sp.nsub):
        d = int(Dm[b])
        s += u[b][d:d + L]
    nv = L // ds
    return s[: nv * ds].reshape(nv, ds).sum(axis=1)
