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

The NUTS proposal ("nuts"; Sec. V names NUTS beside HMC as the next proposal, without
giving its L-kernel): the trajectory of the same leapfrog (step as above, run backwards in
time by negating the velocity) is doubled in a random direction until it makes a U-turn,
diverges or reaches the maximum depth J (Hoffman and Gelman's no-U-turn criterion: a
sub-trajectory whose end points satisfy (theta+ - theta-) . v < 0 at either end stops the
doubling).  The new point is drawn from the trajectory with multinomial weights exp(-H),
H = -log pi + |v|^2 / (2 gamma^2): uniform progressive sampling inside each new
sub-trajectory and biased progressive sampling when it is merged with the old one.
Reading for the weight (the paper gives no L-kernel for NUTS): by default the NUTS kernel's
own reversal, under which every weight stays unchanged (the move leaves pi(theta) N(v)
invariant, so this is exact for a fixed target); as an option (nuts_unit_weight=False) the
momentum-reversal L-kernel of the HMC move evaluated at the selected point (theta*, v*),
log w += log pi(theta*) - log pi(theta_0) + |v_0|^2/(2 gamma^2) - |v*|^2/(2 gamma^2), which
carries information but is not the importance weight of the NUTS proposal (the selected
point is a random point of the trajectory, not its deterministic end).  Random numbers:
Philox stream 5 (nuts_draws).
"""
import math

import numpy as np

from . import pf as _pf, normals as _normals, uniform_open as _uniform_open
from . import STREAM_OUTER_XI, STREAM_OUTER_NU, STREAM_NUTS, SYSTEMATIC
from . import philox4x32_10 as _philox, STAT_NAMES as _STAT_NAMES

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


NUTS_DELTA_MAX = 1000.0   # a point with H - H_0 above this is divergent (Hoffman and Gelman)
NUTS_KINDS = ("max_depth", "subtree_uturn", "divergent", "tree_uturn", "not_moved")


def _u_open_word(w):
    """U(0,1] of one 32-bit word: ((w >> 8) + 1) 2^-24."""
    return ((int(w) >> 8) + 1) * 2.0 ** -24


def nuts_draws(seed, k, i, J):
    """The random numbers of one NUTS move of sample i at iteration k (Philox stream 5, the
    sample's key): for doubling j, its direction (+1 if the top bit of word 0 of counter
    (j, 0, 5, 0) is set, else -1) and its merge uniform (word 2 of that counter); for point n
    of doubling j, its selection uniform (word 1 of counter (j, n, 5, 0)).  Points are
    numbered s = 2^j - 1 + n in the order they are built."""
    key = ((seed & 0xFFFFFFFF) ^ (k & 0xFFFFFFFF), ((seed >> 32) ^ i) & 0xFFFFFFFF)
    dirs, u_sel, u_merge = [], [], []
    for j in range(J):
        for n in range(2 ** j):
            w = _philox((j, n, STREAM_NUTS, 0), key)
            if n == 0:
                dirs.append(1 if (w[0] >> 31) else -1)
                u_merge.append(_u_open_word(w[2]))
            u_sel.append(_u_open_word(w[1]))
    return dirs, u_sel, u_merge


def _logaddexp(a, b):
    if a == -np.inf:
        return b
    if b == -np.inf:
        return a
    m = max(a, b)
    return m + math.log1p(math.exp(-abs(a - b)))


def _uturn_margin(d, th_first, v_first, th_last, v_last):
    """No-U-turn criterion of a sub-trajectory built in direction d from th_first to th_last:
    the smaller of (theta+ - theta-) . v at its two ends (negative: a U-turn), and the same
    relative to |theta+ - theta-| |v| (the scale of its rounding)."""
    dth = d * (th_last - th_first)
    a, b = float(dth @ v_first), float(dth @ v_last)
    na = float(np.linalg.norm(dth))
    rel = min(abs(a) / max(na * float(np.linalg.norm(v_first)), 1e-300),
              abs(b) / max(na * float(np.linalg.norm(v_last)), 1e-300))
    return min(a, b), rel


def nuts_move(theta0, v0, lp0, grad0, payload0, point_fn, gamma, J, dirs, u_sel, u_merge,
              hint=None, band_h=1e-3, band_u=1e-3):
    """One NUTS move from (theta0, v0) with log pi(theta0) = lp0, grad log pi(theta0) = grad0.

    point_fn(theta, s) -> (log pi, grad log pi, payload) runs the particle filter at new point s
    (s = 2^j - 1 + n for point n of doubling j); payload (the filter's log-likelihood and
    gradient) travels with the selected point.  The
    random numbers come in as arguments (nuts_draws).  hint: decisions taken elsewhere,
    {"sel": bits, "merge": bits, "stop": (s, kind)}; where this move decides differently, it
    follows the hint when its own decision is within the band (a near-tie) and counts the
    difference as a tie, else counts a mismatch (and still follows, so later steps compare).

    Returns dict(theta, v, lp, payload, ke0, ke_sel, depth, stop=(s, kind), trace, stats)."""
    g2 = gamma * gamma
    half = 0.5 * g2

    def kin(v):
        return 0.5 * float(v @ v) / g2

    stats = {"nuts_ties": 0, "nuts_mismatch": 0, "points": 0}
    trace = {"sel": 0, "merge": 0, "stop": (2 ** J - 2, 0)}
    ke0 = kin(v0)
    sel = {"theta": theta0, "v": v0, "lp": lp0, "payload": payload0}
    if not np.isfinite(lp0) or not np.all(np.isfinite(grad0)):
        trace["stop"] = (-1, 4)
        return dict(sel, ke0=ke0, ke_sel=ke0, depth=0, stop=(-1, 4), trace=trace, stats=stats)
    H0 = -lp0 + ke0

    def decide(own, key, margin, band):
        """own decision, or the hint's where they differ (tie if |margin| < band)"""
        if hint is None or key is None:
            return own
        other = key
        if other != own:
            stats["nuts_ties" if abs(margin) < band else "nuts_mismatch"] += 1
        return other

    def gpu_stops(s, kind):
        if hint is None:
            return None
        hs, hk = hint["stop"]
        return hs == s and hk == kind

    lsw = -H0
    ends = {+1: (theta0, v0, grad0), -1: (theta0, v0, grad0)}
    depth = 0
    for j in range(J):
        d = dirs[j]
        th_f, v_f, g_f = ends[d]
        lsw_sub = -np.inf
        cand = None
        ck = {}
        stopped = None
        for n in range(2 ** j):
            s = 2 ** j - 1 + n
            # one leapfrog step in direction d from the frontier
            vh = v_f + d * half * g_f
            th = th_f + d * vh
            lp, g, payload = point_fn(th, s)
            stats["points"] += 1
            broken = not (np.isfinite(lp) and np.all(np.isfinite(g)))
            v = vh + d * half * g if not broken else vh
            H = -lp + kin(v) if not broken else np.inf
            own = broken or (H - H0 > NUTS_DELTA_MAX)
            if decide(own, gpu_stops(s, 2), np.inf if broken else (H - H0 - NUTS_DELTA_MAX), band_h):
                stopped = (s, 2)
                break
            # uniform progressive sampling inside the sub-trajectory
            lsw_new = _logaddexp(lsw_sub, -H)
            m = (-H - lsw_new) - math.log(u_sel[s])
            hbit = None if hint is None else bool((hint["sel"] >> s) & 1)
            if decide(m >= 0.0, hbit, m, band_h):
                cand = {"theta": th, "v": v, "lp": lp, "payload": payload}
                trace["sel"] |= 1 << s
            lsw_sub = lsw_new
            # no-U-turn checks of the completed blocks of 2, 4, ... points of this doubling
            uturn, rel = False, np.inf
            for l in range(1, j + 1):
                if n % (2 ** l) == 0:
                    ck[l] = (th, v)
                if (n + 1) % (2 ** l) == 0:
                    mg, r = _uturn_margin(d, ck[l][0], ck[l][1], th, v)
                    if mg < 0.0:
                        uturn = True
                    rel = min(rel, r)
            if decide(uturn, gpu_stops(s, 1), rel, band_u):
                stopped = (s, 1)
                break
            th_f, v_f, g_f = th, v, g
        if stopped is not None:
            trace["stop"] = stopped
            break
        # biased progressive sampling: the new sub-trajectory's candidate replaces the
        # selected point with probability min(1, W_new / W_old)
        m = (lsw_sub - lsw) - math.log(u_merge[j])
        hbit = None if hint is None else bool((hint["merge"] >> j) & 1)
        if decide(m >= 0.0, hbit, m, band_h):
            sel = cand
            trace["merge"] |= 1 << j
        lsw = _logaddexp(lsw, lsw_sub)
        ends[d] = (th_f, v_f, g_f)
        depth = j + 1
        s_last = 2 ** (j + 1) - 2
        mg, rel = _uturn_margin(+1, ends[-1][0], ends[-1][1], ends[+1][0], ends[+1][1])
        if decide(mg < 0.0, gpu_stops(s_last, 3), rel, band_u):
            trace["stop"] = (s_last, 3)
            break
    return dict(sel, ke0=ke0, ke_sel=kin(sel["v"]), depth=depth, stop=trace["stop"], trace=trace,
                stats=stats)


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
    failed; (NUTS): the per-sample weight correction of the move (nuts_step)."""
    N = state.logw.shape[0]
    lp_new = log_prior(theta_new, m0, s0, prior_kind) + ll_new
    gp_new = grad_log_prior(theta_new, m0, s0, prior_kind) + g_new
    if k == 1:
        # w_1 = pi/q_1 = p-hat(y|theta) (Eq. init_weights)
        logw = ll_new.copy()
    elif proposal == "nuts":
        # kinetic = (|v_0|^2/(2 gamma^2) - |v*|^2/(2 gamma^2) per sample, unit): the momentum
        # reversal at the selected point, or (unit) the NUTS kernel's own reversal, which
        # leaves the weight unchanged
        corr, unit = kinetic
        ok = (state.logw > -np.inf) & (lp_new > -np.inf) & (state.logpi > -np.inf)
        with np.errstate(invalid="ignore", over="ignore"):
            moved = state.logw if unit else state.logw + lp_new - state.logpi + corr
            logw = np.where(ok, moved, -np.inf)
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
    grad_ok = np.all(np.isfinite(gp_new), axis=1) if proposal in ("langevin", "hmc", "nuts") else np.ones(N, bool)
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
        prior_kind=GAUSSIAN_PRIOR, hmc_steps=1, nuts_depth=3, nuts_unit_weight=True):
    """Run K iterations; returns (list of per-iteration records, recycled mean).

    proposal: "rw" (SMC0), "langevin" (SMC1), "hmc" (hmc_steps leapfrog steps; the hints,
      when given, apply to the filters at the last leapfrog point) or "nuts" (trajectories of
      at most 2^nuts_depth - 1 new points; hints may carry "nuts": per sample
      {"sel", "merge", "stop"} decisions, followed at near-ties).
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
        elif proposal == "nuts" and k > 1:
            theta_new, ll_new, g_new, kinetic, pfstats, pfrows, nuts_rec = nuts_step(
                state, k, seed, gamma, nuts_depth, nuts_unit_weight, family, dx, dy, H, y, M, scheme,
                ess_frac, band, flag_band, band_rel, loglik_grad_fn, m0, s0, prior_kind, hint)
        else:
            theta_new = propose(state, k, seed, gamma, proposal, m0, s0, prior_kind)
            ll_new, g_new, pfstats, pfrows = run_filters(family, dx, dy, H, y, M, seed, k, theta_new,
                                                         range(N), scheme, ess_frac, hint, band, flag_band,
                                                         band_rel, loglik_grad_fn)
        rec = update(state, k, theta_new, ll_new, g_new, seed, gamma, proposal, m0, s0, hint,
                     outer_band, outer_flag_band, prior_kind, kinetic)
        rec["pf_stats"] = pfstats
        rec["pf_stats_rows"] = pfrows
        if proposal == "nuts" and k > 1:
            rec["nuts"] = nuts_rec
        records.append(rec)
    return records, recycled_mean(records)


def nuts_step(state, k, seed, gamma, J, unit_weight, family, dx, dy, H, y, M, scheme, ess_frac,
              band, flag_band, band_rel, loglik_grad_fn, m0, s0, prior_kind, hint=None):
    """The NUTS move of every sample at iteration k > 1, one sample after the other: momentum
    v_0 = gamma xi (xi from Philox stream 3, as the HMC move), the sample's particle filter
    (its own CRN key) at every new trajectory point, the move of nuts_move.  Returns the
    selected points, their filter outputs, (the kinetic-energy differences
    |v_0|^2/(2 gamma^2) - |v*|^2/(2 gamma^2), unit_weight) for the weight (update), aggregated and
    per-row filter statistics, and per-sample records (depth, stop, trace, stats).  hint: optional
    {"nuts": per-sample move decisions (nuts_move), "nuts_pf": per point s, (pf_anc [N][T][M],
    pf_flag [N][T]) of the filters run elsewhere at that point} -- followed at near-ties only."""
    N, D = state.theta.shape
    move_hints = hint.get("nuts") if hint is not None else None
    pf_hints = hint.get("nuts_pf") if hint is not None else None
    xi = hmc_xi(state, k, seed)
    theta_new = np.empty_like(state.theta)
    ll_new = np.empty(N)
    g_new = np.empty((N, D))
    corr = np.empty(N)
    agg, rows, recs = {}, [], []
    for i in range(N):
        row_stats = {}

        def point_fn(th, s, i=i, row_stats=row_stats):
            if loglik_grad_fn is not None:
                ll, g = loglik_grad_fn(th)
            else:
                ha = hf = None
                if pf_hints is not None:
                    ha, hf = pf_hints[s][0][i], pf_hints[s][1][i]
                out = _pf(family, dx, dy, H, th, y, M, seed, k, i, scheme=scheme, ess_frac=ess_frac,
                          want_grad=True, hint_anc=ha, hint_flag=hf, band=band, flag_band=flag_band,
                          want_tape=False, band_rel=band_rel)
                ll, g = out["loglik"], out["grad"]
                for key, v in out["stats"].items():
                    row_stats[key] = row_stats.get(key, 0) + v
            lp = float(log_prior(th, m0, s0, prior_kind)) + ll
            gp = grad_log_prior(th, m0, s0, prior_kind) + g
            return lp, gp, (ll, np.asarray(g, dtype=np.float64))

        dirs, u_sel, u_merge = nuts_draws(seed, k, i, J)
        th0 = state.theta[i]
        g0 = state.gradpi[i] - grad_log_prior(th0, m0, s0, prior_kind)
        res = nuts_move(th0, gamma * xi[i], state.logpi[i], state.gradpi[i], (state.loglik[i], g0),
                        point_fn, gamma, J, dirs, u_sel, u_merge,
                        hint=move_hints[i] if move_hints is not None else None)
        theta_new[i] = res["theta"]
        ll_new[i], g_new[i] = res["payload"]
        corr[i] = res["ke0"] - res["ke_sel"]
        for key in _STAT_NAMES:
            row_stats.setdefault(key, 0)
        rows.append(row_stats)
        for key, v in row_stats.items():
            agg[key] = agg.get(key, 0) + v
        recs.append({"depth": res["depth"], "stop": res["stop"], "trace": res["trace"], "stats": res["stats"]})
    return theta_new, ll_new, g_new, (corr, bool(unit_weight)), agg, rows, recs


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
        if hint is not None and "pf_anc" in hint:
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
