"""Outer SMC^2 sampler of Sec. III in FP64 numpy (test infrastructure only).

One iteration k, in the order used throughout this project:
  propose (Eq. proposal; SMC0 random walk or SMC1 Langevin of Sec. III-D)
  -> CRN particle filter per sample (the C oracle, key (seed^k, seed_hi^i))
  -> weight (Eq. l_weights with the Langevin L-kernel of Sec. III-E)
  -> normalise (Eq. normalise_smc2) -> estimate (Eq. realised_estimates)
  -> recycling statistic l_k (Eq. recycling_I) -> ESS (Eq. ess_smc2)
  -> systematic resampling when ESS < N/2 (Sec. III-B), sum of weights kept.
Iteration 1 draws theta from the prior q_1 and weights by pi/q_1, i.e. by the
estimated likelihood (Eqs. init_sample, init_weights).

Readings where the paper is silent or inconsistent:
  * Langevin drift F(theta) = 0.5 gamma^2 grad log pi(theta) (the definition of
    F in Sec. III-D; the later display without the 1/2 is not used);
  * L(theta_{k-1}|theta_k) = N(theta_{k-1}; theta_k + F(theta_k), gamma^2 I),
    the one-step leapfrog reversal, so the weight is the MALA ratio used as an
    importance weight with no accept/reject;
  * log pi-hat and its gradient travel with each sample through resampling;
  * the prior is N(prior_mean, diag(prior_std^2)).

The HMC proposal (the extension Sec. V names, "hmc"): L leapfrog steps of Hamiltonian
dynamics whose single step is the SMC1 move above (Sec. III-D notes that Langevin is HMC
with one step).  In displacement form the momentum is v ~ N(0, gamma^2 I) with kinetic
energy |v|^2 / (2 gamma^2), and each step is v += F(theta); theta += v; v += F(theta).
The L-kernel that reverses the momentum weights the end point by
pi(theta_L) N(v_L; 0, gamma^2 I) / (pi(theta_0) N(v_0; 0, gamma^2 I)); with L = 1 this is
the Langevin weight above.  Every leapfrog point runs the particle filters with the
iteration's CRN keys.
"""
import math

import numpy as np

from . import pf as _pf, normals as _normals, uniform_open as _uniform_open
from . import STREAM_OUTER_XI, STREAM_OUTER_NU, SYSTEMATIC

LOG_2PI = np.log(2.0 * np.pi)


GAUSSIAN_PRIOR = 0
UNIFORM_PRIOR = 1


def log_prior(theta, m, s, kind=GAUSSIAN_PRIOR):
    """Gaussian N(m, diag(s^2)), or (kind UNIFORM_PRIOR) uniform on the box [m, s] (Sec. IV-A:
    uniform priors), -inf outside it."""
    if kind == UNIFORM_PRIOR:
        inside = np.all((theta >= m) & (theta <= s), axis=-1)
        return np.where(inside, -np.sum(np.log(s - m)), -np.inf)
    z = (theta - m) / s
    return np.sum(-0.5 * z * z - np.log(s) - 0.5 * LOG_2PI, axis=-1)


def grad_log_prior(theta, m, s, kind=GAUSSIAN_PRIOR):
    if kind == UNIFORM_PRIOR:
        return np.zeros_like(theta)
    return -(theta - m) / (s * s)


def _std_normal_cdf(z):
    return 0.5 * np.vectorize(math.erfc)(-z / math.sqrt(2.0))


def log_normal_iso(x, mean, gamma):
    D = x.shape[-1]
    d = x - mean
    return -0.5 * np.sum(d * d, axis=-1) / (gamma * gamma) - D * np.log(gamma) - 0.5 * D * LOG_2PI


def _lse(v):
    m = np.max(v)
    return m + np.log(np.sum(np.exp(v - m)))


def systematic_ancestors(logw, nu, hint=None, band=1e-6):
    """Systematic ancestors a_i = min{j : c_j >= (i + nu)/N} with follow-mode accounting."""
    N = logw.shape[0]
    w = np.exp(logw - _lse(logw))
    c = np.cumsum(w)
    c = c / c[-1]
    c[-1] = 1.0
    tau = (np.arange(N) + nu) / N
    own = np.searchsorted(c, tau, side="left")           # first j with c_j >= tau
    own = np.minimum(own, N - 1)
    stats = {"near_ties": 0, "tie_followed": 0, "nontie_mismatch": 0}
    a = own.copy()
    for i in range(N):
        j = own[i]
        if (c[j] - tau[i] < band) or (j > 0 and tau[i] - c[j - 1] <= band):
            stats["near_ties"] += 1
        if hint is not None and int(hint[i]) != j:
            h = int(hint[i])
            lo = c[h - 1] if h > 0 else 0.0
            dist = max(tau[i] - c[h], lo - tau[i])
            if dist < band:
                stats["tie_followed"] += 1
            else:
                stats["nontie_mismatch"] += 1
            a[i] = h
    return a, stats


class State:
    """Outer-sampler state of N samples (all FP64): theta [N][D], log w, log pi-hat,
    grad log pi, log p-hat."""

    def __init__(self, N, D):
        self.theta = np.zeros((N, D))
        self.logw = np.zeros(N)
        self.logpi = np.zeros(N)
        self.gradpi = np.zeros((N, D))
        self.loglik = np.zeros(N)


def leapfrog(theta, v, gradpi, L, gamma, grad_fn):
    """L leapfrog steps from (theta, v) with grad log pi(theta) = gradpi, in displacement
    form (force F = 0.5 gamma^2 grad log pi): v += F; theta += v; v += F.  grad_fn(theta, l)
    returns (log pi, grad log pi) at the l-th new point (l = 0 .. L-1).  Returns the end
    point, its momentum, log pi and gradient, and the log pi of every point visited."""
    half = 0.5 * gamma * gamma
    lps = []
    lp = None
    for l in range(L):
        v = v + half * gradpi
        theta = theta + v
        lp, gradpi = grad_fn(theta, l)
        lps.append(lp)
        v = v + half * gradpi
    return theta, v, lp, gradpi, lps


def hmc_xi(state, k, seed):
    """The momentum normals of iteration k (Philox stream 3, as the SMC0/SMC1 moves)."""
    N, D = state.theta.shape
    return np.stack([_normals(seed, k, i, 0, STREAM_OUTER_XI, D) for i in range(N)])


def propose(state, k, seed, gamma, proposal, m0, s0, prior_kind=GAUSSIAN_PRIOR):
    """theta' for iteration k: a prior draw at k = 1 (Eq. init_sample; a uniform prior maps the
    normal xi through its CDF), else the random-walk (SMC0) or Langevin (SMC1) move of
    Sec. III-D with normals from Philox stream 3."""
    N, D = state.theta.shape
    xi = np.stack([_normals(seed, k, i, 0, STREAM_OUTER_XI, D) for i in range(N)])
    if k == 1:
        if prior_kind == UNIFORM_PRIOR:
            return m0 + (s0 - m0) * _std_normal_cdf(xi)
        return m0 + s0 * xi
    drift = 0.5 * gamma * gamma * state.gradpi if proposal == "langevin" else np.zeros_like(state.gradpi)
    return state.theta + drift + gamma * xi


def update(state, k, theta_new, ll_new, g_new, seed, gamma, proposal, m0, s0, hint=None,
           outer_band=1e-4, outer_flag_band=1e-3, prior_kind=GAUSSIAN_PRIOR, kinetic=None):
    """Complete iteration k from the filter outputs at theta_new: weight, normalise,
    estimate, recycling statistic, ESS, resampling.  Updates state; returns the record.
    kinetic (HMC): (|v_0|^2, |v_L|^2) / (2 gamma^2) per sample, NaN where a leapfrog point
    failed."""
    N = state.logw.shape[0]
    lp_new = log_prior(theta_new, m0, s0, prior_kind) + ll_new
    gp_new = grad_log_prior(theta_new, m0, s0, prior_kind) + g_new
    if k == 1:
        # w_1 = pi/q_1 = p-hat(y|theta) (Eq. init_weights)
        logw = ll_new.copy()
    elif proposal == "hmc":
        # momentum-reversal L-kernel: pi(theta_L) N(v_L) / (pi(theta_0) N(v_0))
        ke0, keL = kinetic
        ok = (state.logw > -np.inf) & (lp_new > -np.inf) & (state.logpi > -np.inf)
        with np.errstate(invalid="ignore", over="ignore"):
            logw = np.where(ok, state.logw + lp_new - state.logpi + ke0 - keL, -np.inf)
    else:
        if proposal == "langevin":
            drift = 0.5 * gamma * gamma * state.gradpi
            drift_new = 0.5 * gamma * gamma * gp_new
        else:
            drift = np.zeros_like(state.gradpi)
            drift_new = np.zeros_like(gp_new)
        log_q = log_normal_iso(theta_new, state.theta + drift, gamma)     # q(theta_k | theta_{k-1})
        log_L = log_normal_iso(state.theta, theta_new + drift_new, gamma)  # L(theta_{k-1} | theta_k)
        # Eq. l_weights; a sample whose weight or posterior estimate (old or new) is zero
        # keeps weight zero (this also covers proposals outside a uniform prior's support)
        ok = (state.logw > -np.inf) & (lp_new > -np.inf) & (state.logpi > -np.inf)
        with np.errstate(invalid="ignore", over="ignore"):
            logw = np.where(ok, state.logw + lp_new - state.logpi + log_L - log_q, -np.inf)
    # The Langevin kernels (the SMC1 proposal of Sec. III-D, the L-kernel of Sec. III-E) need
    # grad log pi at the proposal.  Where it is not finite the sample can neither be
    # weighted nor moved: it carries weight zero, as does any non-finite weight.
    grad_ok = np.all(np.isfinite(gp_new), axis=1) if proposal in ("langevin", "hmc") else np.ones(N, bool)
    logw = np.where(grad_ok & np.isfinite(logw), logw, -np.inf)
    theta, logpi, gradpi, loglik = theta_new, lp_new, gp_new, ll_new

    # normalise, estimate (over the samples of positive weight), recycling statistic, ESS
    L = _lse(logw)
    wn = np.exp(logw - L)
    pos = wn > 0.0
    mean = wn[pos] @ theta[pos]
    ess = 1.0 / np.sum(wn * wn)
    l_k = np.exp(2.0 * _lse(logw) - _lse(2.0 * logw))        # (sum w)^2 / sum w^2
    rec = {"k": k, "ess": float(ess), "l_k": float(l_k), "mean": mean.copy(),
           "theta": theta.copy(), "logw": logw.copy(), "loglik": loglik.copy(),
           "grad": gradpi.copy(), "resampled": False, "outer_stats": {}}
    own_flag = ess < N / 2.0
    flag = own_flag
    if hint is not None and "outer_flag" in hint and bool(hint["outer_flag"]) != own_flag:
        near = abs(ess / (N / 2.0) - 1.0) < outer_flag_band
        rec["outer_stats"]["flag_tie" if near else "flag_disagree"] = 1
        flag = bool(hint["outer_flag"])
    if flag:
        nu = _uniform_open(seed, k, 0, 0, STREAM_OUTER_NU)
        hint_a = hint["outer_anc"] if (hint is not None and "outer_anc" in hint) else None
        a, st = systematic_ancestors(logw, nu, hint_a, band=outer_band)
        rec["outer_stats"].update(st)
        rec["ancestors"] = a
        theta, logpi, gradpi, loglik = theta[a], logpi[a], gradpi[a], loglik[a]
        logw = np.full(N, L - np.log(N))
        rec["resampled"] = True
    state.theta, state.logw, state.logpi, state.gradpi, state.loglik = theta, logw, logpi, gradpi, loglik
    return rec


def recycled_mean(records):
    """Sec. III-C: sum_k c_k f~_k with c_k = l_k / sum_k l_k (Eq. opt_recycling_constant)."""
    lks = np.array([r["l_k"] for r in records])
    ck = lks / lks.sum()
    return sum(c * r["mean"] for c, r in zip(ck, records))


def run(family, dx, dy, H, y, N, M, K, gamma, proposal, seed, prior_mean=None, prior_std=None,
        scheme=SYSTEMATIC, ess_frac=0.5, hints=None, band=1e-6, flag_band=1e-6,
        outer_band=1e-4, D=None, loglik_grad_fn=None, band_rel=0.0, outer_flag_band=1e-3,
        prior_kind=GAUSSIAN_PRIOR, hmc_steps=1):
    """Run K iterations; returns (list of per-iteration records, recycled mean).

    proposal: "rw" (SMC0), "langevin" (SMC1) or "hmc" (hmc_steps leapfrog steps; the hints,
      when given, apply to the filters at the last leapfrog point).
    hints: optional list, per iteration, of dicts with keys pf_anc (N,T,M), pf_flag (N,T),
      outer_anc (N,), outer_flag (bool): decisions taken elsewhere, followed at near-ties
      (PF level: |c - tau| < band; outer level: |c - tau| < outer_band, and the resampling
      decision when |ESS/(N/2) - 1| < outer_flag_band).
    loglik_grad_fn: optional theta -> (log p, grad) used in place of the particle filter
      (e.g. the exact Kalman likelihood, to test the sampler on its own).
    """
    if D is None:
        D = 3 if family in (1, 2) else 2 * dx + dy
    m0 = np.zeros(D) if prior_mean is None else np.asarray(prior_mean, dtype=np.float64)
    s0 = np.ones(D) if prior_std is None else np.asarray(prior_std, dtype=np.float64)
    seed = int(seed)
    records = []
    state = State(N, D)
    for k in range(1, K + 1):
        hint = hints[k - 1] if hints is not None else None
        kinetic = None
        if proposal == "hmc" and k > 1:
            L = int(hmc_steps)
            last = {}

            def grad_fn(th, l):
                ll, g, st, rows = run_filters(family, dx, dy, H, y, M, seed, k, th, range(N), scheme,
                                              ess_frac, hint if l == L - 1 else None, band, flag_band,
                                              band_rel, loglik_grad_fn)
                last.update(ll=ll, g=g, st=st, rows=rows)
                lp = log_prior(th, m0, s0, prior_kind) + ll
                gp = grad_log_prior(th, m0, s0, prior_kind) + g
                # a point whose estimate or gradient is not finite breaks the trajectory
                bad = ~(np.isfinite(lp) & np.all(np.isfinite(gp), axis=1))
                last["bad"] = last.get("bad", np.zeros(N, bool)) | bad
                return lp, gp

            xi = hmc_xi(state, k, seed)
            theta_new, vL, _, _, _ = leapfrog(state.theta, gamma * xi, state.gradpi, L, gamma, grad_fn)
            ll_new, g_new, pfstats, pfrows = last["ll"], last["g"], last["st"], last["rows"]
            ke0 = 0.5 * np.sum(xi * xi, axis=1)
            with np.errstate(invalid="ignore", over="ignore"):
                keL = 0.5 * np.sum(vL * vL, axis=1) / (gamma * gamma)
            keL = np.where(last["bad"], np.nan, keL)
            kinetic = (ke0, keL)
        else:
            theta_new = propose(state, k, seed, gamma, proposal, m0, s0, prior_kind)
            ll_new, g_new, pfstats, pfrows = run_filters(family, dx, dy, H, y, M, seed, k, theta_new,
                                                         range(N), scheme, ess_frac, hint, band, flag_band,
                                                         band_rel, loglik_grad_fn)
        rec = update(state, k, theta_new, ll_new, g_new, seed, gamma, proposal, m0, s0, hint,
                     outer_band, outer_flag_band, prior_kind, kinetic)
        rec["pf_stats"] = pfstats
        rec["pf_stats_rows"] = pfrows
        records.append(rec)
    return records, recycled_mean(records)


def run_filters(family, dx, dy, H, y, M, seed, k, theta, rows, scheme=SYSTEMATIC, ess_frac=0.5,
                hint=None, band=1e-6, flag_band=1e-6, band_rel=0.0, loglik_grad_fn=None):
    """CRN particle filters (forward-mode gradient) of the given rows of theta with the
    Philox keys of those rows; returns (log p-hat, gradient, aggregated stats, per-row stats)."""
    rows = list(rows)
    D = theta.shape[1]
    ll = np.zeros(len(rows))
    g = np.zeros((len(rows), D))
    agg = {}
    stats_rows = []
    for r, i in enumerate(rows):
        if loglik_grad_fn is not None:
            ll[r], g[r] = loglik_grad_fn(theta[i])
            continue
        ha = hf = None
        if hint is not None:
            ha = hint["pf_anc"][i]
            hf = hint["pf_flag"][i]
        out = _pf(family, dx, dy, H, theta[i], y, M, seed, k, i, scheme=scheme,
                  ess_frac=ess_frac, want_grad=True, hint_anc=ha, hint_flag=hf,
                  band=band, flag_band=flag_band, want_tape=False, band_rel=band_rel)
        ll[r] = out["loglik"]
        g[r] = out["grad"]
        stats_rows.append(out["stats"])
        for key, v in out["stats"].items():
            agg[key] = agg.get(key, 0) + v
    return ll, g, agg, stats_rows
