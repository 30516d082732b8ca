"""Pins of the oracle's particle filter and Kalman filter (CPU only).

Each test ties the oracle to something other than itself: the exact Kalman
likelihood (itself pinned to the brute-force joint Gaussian density), the
closed form at M=1, the definition of the ancestor index of App. B written
as a count, the unbiasedness of the likelihood estimate (Sec. II-C), central
finite differences of the fixed-tape likelihood, and the Kalman gradient when
resampling is switched off (plain reparameterised importance sampling, which
is consistent).
"""
import numpy as np
import pytest
from scipy import stats

import oracle
import oracle.kalman as kalman
from paper_2407_17296_gb300 import workloads as W


def _lg(w, th):
    return dict(family=oracle.LG_DIAG, dx=w.dx, dy=w.dy, H=w.H, theta=th, y=w.y)


# --------------------------------------------------------------------------- Kalman

@pytest.mark.parametrize("make,T", [(W.lg1, 7), (W.lg4, 4), (W.lg16, 2)])
def test_kalman_matches_joint_gaussian(make, T):
    w = make(T=T)
    th = W.thetas_near(w, 1, 0.1)[0]
    ll, _ = kalman.loglik_grad(th, w.y, w.H, w.dx, w.dy)
    assert ll == pytest.approx(kalman.joint_loglik(th, w.y, w.H, w.dx, w.dy), abs=1e-9)


@pytest.mark.parametrize("make", [W.lg1, W.lg4])
def test_kalman_gradient_matches_fd(make):
    w = make(T=40)
    th = W.thetas_near(w, 1, 0.1)[0]
    _, g = kalman.loglik_grad(th, w.y, w.H, w.dx, w.dy)
    h = 1e-5
    for d in range(w.D):
        e = np.zeros(w.D)
        e[d] = h
        fd = (kalman.loglik_grad(th + e, w.y, w.H, w.dx, w.dy)[0]
              - kalman.loglik_grad(th - e, w.y, w.H, w.dx, w.dy)[0]) / (2 * h)
        assert g[d] == pytest.approx(fd, rel=1e-6, abs=1e-6)


# --------------------------------------------------------------------------- M = 1

def _path_loglik_lg(w, th, seed, it, row):
    """Single-particle path from the shared generator; log p-hat = sum_t log g(y_t|x_t)."""
    dx, dy = w.dx, w.dy
    a, q, r = th[:dx], np.exp(th[dx:2 * dx]), np.exp(th[2 * dx:])
    H = np.eye(dy, dx) if w.H is None else w.H.astype(np.float64)
    x = oracle.normals(seed, it, row, 0, oracle.STREAM_INIT, dx)
    tot = 0.0
    for t in range(1, w.T + 1):
        x = a * x + q * oracle.normals(seed, it, row, t, oracle.STREAM_PROP, dx)
        tot += stats.multivariate_normal.logpdf(w.y[t - 1].astype(np.float64), H @ x, np.diag(r * r))
    return tot


def _path_loglik_sv(w, th, seed, it, row):
    mu, phi, sig = th[0], np.tanh(th[1]), np.exp(th[2])
    x = mu + sig / np.sqrt(1 - phi * phi) * oracle.normals(seed, it, row, 0, oracle.STREAM_INIT, 1)[0]
    tot = 0.0
    for t in range(1, w.T + 1):
        x = mu + phi * (x - mu) + sig * oracle.normals(seed, it, row, t, oracle.STREAM_PROP, 1)[0]
        tot += stats.norm.logpdf(float(w.y[t - 1, 0]), 0.0, np.exp(0.5 * x))
    return tot


@pytest.mark.parametrize("make", [W.lg1, W.lg4, W.lg16])
def test_single_particle_is_path_density_lg(make):
    w = make(T=25)
    th = W.thetas_near(w, 1, 0.1)[0]
    r = oracle.pf(w.family, w.dx, w.dy, w.H, th, w.y, 1, 11, 2, 3)
    assert r["loglik"] == pytest.approx(_path_loglik_lg(w, th, 11, 2, 3), abs=1e-9)


def test_single_particle_is_path_density_sv():
    w = W.sv(T=40)
    th = W.thetas_near(w, 1, 0.1)[0]
    r = oracle.pf(w.family, 1, 1, None, th, w.y, 1, 5, 1, 9)
    assert r["loglik"] == pytest.approx(_path_loglik_sv(w, th, 5, 1, 9), abs=1e-9)


# --------------------------------------------------------------------------- unbiasedness

@pytest.mark.parametrize("scheme", [oracle.SYSTEMATIC, oracle.MULTINOMIAL])
def test_likelihood_estimate_unbiased_vs_kalman(scheme):
    """E[p-hat] = p(y|theta): natural-scale average over seeds within 4.5 standard errors."""
    w = W.lg1(T=4)
    th = np.array([0.7, np.log(0.8), np.log(0.6)])
    ll_kf, _ = kalman.loglik_grad(th, w.y, None, 1, 1)
    n = 6000
    ratios = np.empty(n)
    resampled = 0
    for row in range(n):
        r = oracle.pf(w.family, 1, 1, None, th, w.y, 6, 2024, 1, row, scheme=scheme,
                      want_grad=False, want_tape=False)
        ratios[row] = np.exp(r["loglik"] - ll_kf)
        resampled += r["stats"]["resample_steps"]
    assert resampled > n // 4          # resampling really happened in many runs
    se = ratios.std() / np.sqrt(n)
    assert abs(ratios.mean() - 1.0) < 4.5 * se


def test_likelihood_estimate_unbiased_lg4():
    w = W.lg4(T=3)
    th = w.theta_star
    ll_kf, _ = kalman.loglik_grad(th, w.y, w.H, 4, 2)
    n = 4000
    ratios = np.array([np.exp(oracle.pf(0, 4, 2, w.H, th, w.y, 5, 7, 1, row, want_grad=False,
                                        want_tape=False)["loglik"] - ll_kf) for row in range(n)])
    assert abs(ratios.mean() - 1.0) < 4.5 * ratios.std() / np.sqrt(n)


# --------------------------------------------------------------------------- gradient

@pytest.mark.parametrize("make,T,M", [(W.lg1, 10, 65536), (W.lg4, 8, 32768)])
def test_gradient_consistent_with_kalman_without_resampling(make, T, M):
    w = make(T=T)
    th = w.theta_star
    _, g_kf = kalman.loglik_grad(th, w.y, w.H, w.dx, w.dy)
    rows = 8
    gs = np.array([oracle.pf(w.family, w.dx, w.dy, w.H, th, w.y, M, 31, 1, row, ess_frac=0.0,
                             want_tape=False)["grad"] for row in range(rows)])
    se = gs.std(0, ddof=1) / np.sqrt(rows)
    assert np.all(np.abs(gs.mean(0) - g_kf) < 5 * se + 0.02)


def _fd_replay(w, th, M, tape, flags, h, family=None, seed=13, it=4, row=5):
    fam = w.family if family is None else family
    g = np.zeros(w.D)
    for d in range(w.D):
        e = np.zeros(w.D)
        e[d] = h
        lp = oracle.pf(fam, w.dx, w.dy, w.H, th + e, w.y, M, seed, it, row, want_grad=False,
                       hint_anc=tape, hint_flag=flags, replay=True)["loglik"]
        lm = oracle.pf(fam, w.dx, w.dy, w.H, th - e, w.y, M, seed, it, row, want_grad=False,
                       hint_anc=tape, hint_flag=flags, replay=True)["loglik"]
        g[d] = (lp - lm) / (2 * h)
    return g


@pytest.mark.parametrize("make,T,M", [(W.lg1, 60, 200), (W.lg4, 40, 96), (W.sv, 80, 128),
                                      (W.lg16, 12, 40)])
@pytest.mark.parametrize("scheme", [oracle.SYSTEMATIC, oracle.MULTINOMIAL])
def test_forward_mode_gradient_matches_fd_of_fixed_tape(make, T, M, scheme):
    """App. A/B gradient = derivative of log p-hat with CRN and ancestors held fixed."""
    w = make(T=T)
    th = W.thetas_near(w, 1, 0.05)[0]
    r = oracle.pf(w.family, w.dx, w.dy, w.H, th, w.y, M, 13, 4, 5, scheme=scheme)
    assert r["stats"]["resample_steps"] > 2
    for h in (1e-4, 1e-5):
        fd = _fd_replay(w, th, M, r["anc"], r["flag"], h)
        np.testing.assert_allclose(r["grad"], fd, rtol=2e-5, atol=2e-5 * max(1.0, np.abs(fd).max()))


def test_replay_of_own_tape_is_exact():
    w = W.lg4(T=30)
    th = w.theta_star
    r = oracle.pf(0, 4, 2, w.H, th, w.y, 64, 3, 2, 1)
    rr = oracle.pf(0, 4, 2, w.H, th, w.y, 64, 3, 2, 1, hint_anc=r["anc"], hint_flag=r["flag"],
                   replay=True)
    assert rr["loglik"] == r["loglik"]
    np.testing.assert_array_equal(rr["grad"], r["grad"])
    np.testing.assert_array_equal(rr["anc"], r["anc"])


# --------------------------------------------------------------------------- resampling

def _count_definition(w, tau):
    """App. B: kappa_i = #{j : nu_i > c^j}, 0-based over j = 0..M-2 (c^{M-1} = 1)."""
    c = np.cumsum(w) / np.sum(w)
    return np.array([int(np.sum(t > c[:-1])) for t in tau])


def test_ancestor_definition_random():
    rng = np.random.default_rng(0)
    for M in (1, 2, 3, 7, 64, 1000):
        w = rng.exponential(size=M) * (rng.random(M) < 0.7)
        if w.sum() == 0:
            w[0] = 1.0
        tau = rng.random(257) * (1 - 1e-12) + 1e-12
        np.testing.assert_array_equal(oracle.ancestors(w, tau), _count_definition(w, tau))


def test_ancestor_exact_tie_selects_lower_index():
    # c = (0.25, 0.5, 0.75, 1): a threshold equal to c_j selects j (strict ">" in App. B)
    w = np.ones(4)
    assert list(oracle.ancestors(w, np.array([0.25, 0.5, 0.5000001, 1.0]))) == [0, 1, 2, 3]


def test_systematic_counts_are_floor_or_ceil():
    rng = np.random.default_rng(1)
    for M in (5, 128, 1024):
        w = rng.exponential(size=M) ** 3
        nu = rng.random()
        a = oracle.ancestors(w, (np.arange(M) + nu) / M)
        assert np.all(np.diff(a) >= 0)
        cnt = np.bincount(a, minlength=M)
        assert cnt.sum() == M
        mw = M * w / w.sum()
        assert np.all((cnt >= np.floor(mw) - 1e-9) & (cnt <= np.ceil(mw) + 1e-9))


def _brute_force_pf_lg(w, th, M, seed, it, row, scheme, ess_frac):
    """Tiny-M re-derivation from the paper's definitions with scipy densities."""
    dx, dy = w.dx, w.dy
    a, q, r = th[:dx], np.exp(th[dx:2 * dx]), np.exp(th[2 * dx:])
    H = np.eye(dy, dx) if w.H is None else w.H.astype(np.float64)
    x = oracle.normals(seed, it, row, 0, oracle.STREAM_INIT, M * dx).reshape(M, dx)
    wts = np.ones(M)                   # unnormalised weights, w_0 = 1
    anc_rows, flags = [], []
    for t in range(1, w.T + 1):
        if t > 1:
            wn = wts / wts.sum()
            flag = 1.0 / np.sum(wn * wn) < ess_frac * M
        else:
            flag = False
        flags.append(int(flag))
        if flag:
            if scheme == oracle.SYSTEMATIC:
                nu = oracle.uniform_open(seed, it, row, t, oracle.STREAM_RESAMPLE, 0, 0)
                tau = (np.arange(M) + nu) / M
            else:
                tau = np.array([oracle.uniform_open(seed, it, row, t, oracle.STREAM_RESAMPLE,
                                                    i // 4, i % 4) for i in range(M)])
            kappa = _count_definition(wts, tau)
            x = x[kappa]
            wts = np.full(M, wts.mean())        # Eq. weightresample
            anc_rows.append(kappa)
        else:
            anc_rows.append(np.zeros(M, dtype=int))
        x = a * x + q * oracle.normals(seed, it, row, t, oracle.STREAM_PROP, M * dx).reshape(M, dx)
        g = np.array([stats.multivariate_normal.pdf(w.y[t - 1].astype(np.float64), H @ x[j],
                                                    np.diag(r * r)) for j in range(M)])
        wts = wts * g
    return np.log(wts.mean()), np.array(anc_rows), np.array(flags)


@pytest.mark.parametrize("scheme", [oracle.SYSTEMATIC, oracle.MULTINOMIAL])
@pytest.mark.parametrize("ess_frac", [0.5, 1.0])
@pytest.mark.parametrize("M", [2, 3, 5])
def test_tiny_filter_brute_force(scheme, ess_frac, M):
    w = W.lg4(T=6)
    th = W.thetas_near(w, 1, 0.2)[0]
    ll, anc, flags = _brute_force_pf_lg(w, th, M, 21, 3, 2, scheme, ess_frac)
    r = oracle.pf(0, 4, 2, w.H, th, w.y, M, 21, 3, 2, scheme=scheme, ess_frac=ess_frac)
    np.testing.assert_array_equal(r["flag"], flags)
    np.testing.assert_array_equal(r["anc"][flags == 1], anc[flags == 1])
    assert r["loglik"] == pytest.approx(ll, abs=1e-10)
    if ess_frac == 1.0:
        assert r["stats"]["resample_steps"] == w.T - 1


def test_never_resample_when_fraction_zero():
    w = W.lg4(T=20)
    r = oracle.pf(0, 4, 2, w.H, w.theta_star, w.y, 32, 1, 1, 1, ess_frac=0.0)
    assert r["stats"]["resample_steps"] == 0 and r["flag"].sum() == 0


# --------------------------------------------------------------------------- follow mode

def test_follow_mode_classifies_planted_mismatches():
    w = W.lg4(T=30)
    th = w.theta_star
    M = 64
    r = oracle.pf(0, 4, 2, w.H, th, w.y, M, 3, 1, 0)
    steps = np.nonzero(r["flag"])[0]
    assert len(steps) > 0
    # own tape as hint: nothing to follow
    s = oracle.pf(0, 4, 2, w.H, th, w.y, M, 3, 1, 0, hint_anc=r["anc"], hint_flag=r["flag"])
    assert s["stats"]["nontie_mismatch"] == 0 and s["stats"]["tie_followed"] == 0
    assert s["loglik"] == r["loglik"]
    # plant a far-off ancestor at the last resampled step: a non-tie mismatch, followed
    bad = r["anc"].copy()
    t0 = steps[-1]
    i = M // 2
    bad[t0, i] = (int(bad[t0, i]) + M // 2) % M
    s = oracle.pf(0, 4, 2, w.H, th, w.y, M, 3, 1, 0, hint_anc=bad, hint_flag=r["flag"])
    assert s["stats"]["nontie_mismatch"] == 1 and s["worst"] > 1e-6
    assert s["loglik"] != r["loglik"]
    assert np.array_equal(s["anc"][t0], bad[t0])
    # inside the conditioned band (band_rel * accumulated |log g|) it is counted as such
    s = oracle.pf(0, 4, 2, w.H, th, w.y, M, 3, 1, 0, hint_anc=bad, hint_flag=r["flag"], band_rel=1.0)
    assert s["stats"]["nontie_mismatch"] == 0 and s["stats"]["tie_conditioned"] == 1
    # the same plant inside a huge band counts as a followed tie instead
    s = oracle.pf(0, 4, 2, w.H, th, w.y, M, 3, 1, 0, hint_anc=bad, hint_flag=r["flag"], band=2.0)
    assert s["stats"]["nontie_mismatch"] == 0 and s["stats"]["tie_followed"] == 1
    # a flipped resample flag is a flag mismatch
    f2 = r["flag"].copy()
    f2[t0] = 0
    s = oracle.pf(0, 4, 2, w.H, th, w.y, M, 3, 1, 0, hint_anc=r["anc"], hint_flag=f2)
    assert s["stats"]["flag_mismatch"] >= 1


# --------------------------------------------------------------------------- optimal proposal (Sec. IV-A)

def _lgssm_as_lg1(th):
    """(mu, phi, sigma) -> the LG-diag parameters (a, log q, log r) of the same model."""
    return np.array([th[0], np.log(th[1]), np.log(th[2])])


@pytest.mark.parametrize("scheme", [oracle.SYSTEMATIC, oracle.MULTINOMIAL])
def test_optimal_proposal_estimate_unbiased_vs_kalman(scheme):
    """The optimal proposal's weight p(y_t | x_{t-1}) is right only with its proposal mean and
    variance: together they give an unbiased likelihood estimate (Kalman, 4.5 standard errors)."""
    w = W.lgssm(T=5)
    th = np.array([0.6, 1.3, 0.7])
    ll_kf, _ = kalman.loglik_grad(_lgssm_as_lg1(th), w.y, None, 1, 1)
    n = 5000
    ratios = np.empty(n)
    resampled = 0
    for row in range(n):
        r = oracle.pf(oracle.LG_OPT, 1, 1, None, th, w.y, 6, 77, 1, row, scheme=scheme,
                      ess_frac=1.0, want_grad=False, want_tape=False)
        ratios[row] = np.exp(r["loglik"] - ll_kf)
        resampled += r["stats"]["resample_steps"]
    assert resampled == 4 * n          # every step after the first resampled
    assert abs(ratios.mean() - 1.0) < 4.5 * ratios.std() / np.sqrt(n)


def test_optimal_proposal_single_step_is_exact_in_the_limit():
    """T = 1: the weights p(y_1 | x_0) with x_0 ~ N(0, 1) average to N(y_1; 0, mu^2 + phi^2 + sigma^2)."""
    w = W.lgssm(T=1)
    th = np.array([0.75, 1.0, 1.0])
    r = oracle.pf(oracle.LG_OPT, 1, 1, None, th, w.y, 1 << 16, 5, 1, 0, want_grad=False, want_tape=False)
    exact = stats.norm.logpdf(float(w.y[0, 0]), 0.0, np.sqrt(th[0] ** 2 + th[1] ** 2 + th[2] ** 2))
    assert r["loglik"] == pytest.approx(exact, abs=5e-3)


def test_optimal_proposal_gradient_consistent_with_kalman_without_resampling():
    w = W.lgssm(T=8)
    th = np.array([0.7, 1.1, 0.9])
    _, g_lg1 = kalman.loglik_grad(_lgssm_as_lg1(th), w.y, None, 1, 1)
    g_kf = g_lg1 * np.array([1.0, 1.0 / th[1], 1.0 / th[2]])   # chain rule to (mu, phi, sigma)
    rows = 8
    gs = np.array([oracle.pf(oracle.LG_OPT, 1, 1, None, th, w.y, 1 << 15, 31, 1, row, ess_frac=0.0,
                             want_tape=False)["grad"] for row in range(rows)])
    se = gs.std(0, ddof=1) / np.sqrt(rows)
    assert np.all(np.abs(gs.mean(0) - g_kf) < 5 * se + 0.02)


@pytest.mark.parametrize("scheme", [oracle.SYSTEMATIC, oracle.MULTINOMIAL])
def test_optimal_proposal_gradient_matches_fd_of_fixed_tape(scheme):
    w = W.lgssm(T=60)
    th = np.array([0.7, 1.1, 0.9])
    r = oracle.pf(oracle.LG_OPT, 1, 1, None, th, w.y, 64, 13, 4, 5, scheme=scheme, ess_frac=0.8)
    assert r["stats"]["resample_steps"] > 2
    for h in (1e-4, 1e-5):
        fd = _fd_replay(w, th, 64, r["anc"], r["flag"], h, family=oracle.LG_OPT)
        np.testing.assert_allclose(r["grad"], fd, rtol=2e-5, atol=2e-5 * max(1.0, np.abs(fd).max()))
