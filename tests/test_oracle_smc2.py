"""Pins of the oracle's outer SMC^2 sampler (CPU only).

The random-walk L-kernel ratio is identically one; recycling constants sum to
one and every ESS lies in [1, N]; the systematic outer resampler follows the
count definition; and, with the exact Kalman likelihood in place of the
particle filter, the recycled estimate of both proposals approaches the
posterior mean computed by quadrature.
"""
import numpy as np
import pytest

import oracle
import oracle.kalman as kalman
import oracle.smc2 as smc2
from paper_2407_17296_gb300 import workloads as W


def test_random_walk_l_kernel_ratio_is_one():
    rng = np.random.default_rng(3)
    th0 = rng.standard_normal((50, 5))
    th1 = th0 + 0.3 * rng.standard_normal((50, 5))
    z = np.zeros_like(th0)
    np.testing.assert_array_equal(smc2.log_normal_iso(th0, th1 + z, 0.3),
                                  smc2.log_normal_iso(th1, th0 + z, 0.3))


def test_outer_systematic_ancestors_match_count_definition():
    rng = np.random.default_rng(5)
    for N in (1, 4, 64, 1000):
        logw = rng.standard_normal(N) * 3
        nu = rng.random()
        a, st = smc2.systematic_ancestors(logw, nu)
        w = np.exp(logw - logw.max())
        c = np.cumsum(w) / w.sum()
        want = [int(np.sum((i + nu) / N > c[:-1])) for i in range(N)]
        np.testing.assert_array_equal(a, want)


def _scalar_kf_grid(a, lq, lr, y):
    """Vectorised scalar Kalman log-likelihood over parameter grids (broadcast arrays)."""
    q2, r2 = np.exp(2 * lq), np.exp(2 * lr)
    m = np.zeros(np.broadcast(a, lq, lr).shape)
    P = np.ones_like(m)
    ll = np.zeros_like(m)
    for yt in y.astype(np.float64).ravel():
        mp, Pp = a * m, a * a * P + q2
        S = Pp + r2
        e = yt - mp
        ll += -0.5 * (e * e / S + np.log(S) + np.log(2 * np.pi))
        K = Pp / S
        m, P = mp + K * e, Pp - K * Pp
    return ll


@pytest.mark.parametrize("proposal", ["langevin", "rw"])
def test_sampler_recovers_conjugate_gaussian_posterior(proposal):
    """Exact Gaussian log-likelihood of theta: the posterior is known in closed form.

    The step size (0.4) is large against the posterior spread (~0.29), where an
    unadjusted Langevin move inflates the spread of its stationary law; the
    L-kernel weight must undo that, so the weighted variance pins the weight
    formula (dropping the L-kernel/proposal terms gives ratios of 0.2-0.8)."""
    mu_l = np.array([0.8, -0.5, 0.3])
    s_l = np.array([0.3, 0.4, 0.25])

    def fn(th):
        z = (th - mu_l) / s_l
        return -0.5 * np.sum(z * z), -z / s_l

    prec = 1.0 + 1.0 / s_l ** 2
    post_mean = (mu_l / s_l ** 2) / prec
    post_var = 1.0 / prec
    N = 3000
    recs, rec_mean = smc2.run(0, 1, 1, None, np.zeros((1, 1), np.float32), N, 1, 20, 0.4,
                              proposal, 123, loglik_grad_fn=fn, D=3)
    for r in recs:
        assert 1.0 - 1e-9 <= r["ess"] <= N + 1e-9
    lk = np.array([r["l_k"] for r in recs])
    assert np.isclose((lk / lk.sum()).sum(), 1.0)
    assert np.all(np.abs(rec_mean - post_mean) < 0.1 * np.sqrt(post_var))
    last = recs[-1]
    w = np.exp(last["logw"] - last["logw"].max())
    w /= w.sum()
    var = w @ (last["theta"] - last["mean"]) ** 2
    assert np.all((var / post_var > 0.8) & (var / post_var < 1.3)), var / post_var


def test_sampler_with_exact_lg_likelihood_finds_quadrature_posterior_mean():
    w = W.lg1(T=100)
    ga = np.linspace(0.3, 1.05, 76)
    gq = np.linspace(np.log(0.1), np.log(1.6), 76)
    gr = np.linspace(np.log(0.4), np.log(1.6), 76)
    A, Q, R = np.meshgrid(ga, gq, gr, indexing="ij")
    lp = _scalar_kf_grid(A, Q, R, w.y) - 0.5 * (A * A + Q * Q + R * R)
    p = np.exp(lp - lp.max())
    p /= p.sum()
    post = np.array([(p * A).sum(), (p * Q).sum(), (p * R).sum()])
    post_sd = np.sqrt(np.array([(p * A * A).sum(), (p * Q * Q).sum(), (p * R * R).sum()]) - post ** 2)

    def fn(th):
        return kalman.loglik_grad(th, w.y, None, 1, 1)

    recs, _ = smc2.run(w.family, 1, 1, None, w.y, 128, 1, 12, 0.06, "langevin", 99,
                       loglik_grad_fn=fn)
    final = recs[-1]["mean"]
    assert np.all(np.abs(final - post) < 0.5 * post_sd + 0.02), (final, post, post_sd)


def test_sampler_with_particle_filter_runs_and_keeps_invariants():
    w = W.lg1(T=30)
    recs, rec_mean = smc2.run(w.family, 1, 1, None, w.y, 16, 32, 4, 0.2, "langevin", 5)
    assert len(recs) == 4
    for r in recs:
        assert 1.0 - 1e-9 <= r["ess"] <= 16 + 1e-9
        assert np.all(np.isfinite(r["theta"])) and np.all(np.isfinite(r["grad"]))
    assert np.all(np.isfinite(rec_mean))


def test_sampler_with_uniform_prior_finds_quadrature_posterior_mean():
    """Sec. IV-A's model and uniform priors, exact likelihood: the recycled estimate after the
    run lies near the posterior mean computed by quadrature over the prior's box."""
    from oracle import kalman
    w = W.lgssm(T=60)
    gm = np.linspace(0.2, 0.99, 60)
    gp = np.linspace(0.3, 2.0, 60)
    gs = np.linspace(0.3, 2.0, 60)
    A, P, S = np.meshgrid(gm, gp, gs, indexing="ij")
    lp = _scalar_kf_grid(A, np.log(P), np.log(S), w.y)   # flat prior inside the box
    p = np.exp(lp - lp.max())
    p /= p.sum()
    post = np.array([(p * A).sum(), (p * P).sum(), (p * S).sum()])
    post_sd = np.sqrt(np.array([(p * A * A).sum(), (p * P * P).sum(), (p * S * S).sum()]) - post ** 2)

    def fn(th):
        if th[1] <= 0.0 or th[2] <= 0.0:
            return -np.inf, np.zeros(3)
        ll, g = kalman.loglik_grad(np.array([th[0], np.log(th[1]), np.log(th[2])]), w.y, None, 1, 1)
        return ll, g * np.array([1.0, 1.0 / th[1], 1.0 / th[2]])

    recs, rec_mean = smc2.run(w.family, 1, 1, None, w.y, 256, 1, 15, 0.05, "langevin", 5,
                              prior_mean=w.prior_mean, prior_std=w.prior_std, D=3,
                              loglik_grad_fn=fn, prior_kind=smc2.UNIFORM_PRIOR)
    final = recs[-1]["mean"]
    assert np.all(np.abs(final - post) < 0.5 * post_sd + 0.03), (final, post, post_sd)
    # every draw of iteration 1 lies inside the box
    th1 = recs[0]["theta"]
    assert np.all((th1 >= w.prior_mean) & (th1 <= w.prior_std))


@pytest.mark.parametrize("k", [1, 2])
def test_nonfinite_gradient_or_weight_gets_zero_weight(k):
    """A proposal whose filter gradient overflowed (finite log p-hat, non-finite gradient)
    cannot be moved by the Langevin kernel or weighted by its L-kernel: it gets weight zero,
    and neither it nor a NaN state of a zero-weight sample reaches the estimate."""
    rng = np.random.default_rng(11)
    N, D = 8, 3
    st = smc2.State(N, D)
    st.theta = rng.standard_normal((N, D))
    st.gradpi = rng.standard_normal((N, D))
    st.logpi = rng.standard_normal(N)
    st.logw = np.zeros(N)
    th_new = st.theta + 0.1 * rng.standard_normal((N, D))
    th_new[5] = np.nan  # a zero-weight sample's state may be anything
    ll_new = -np.abs(rng.standard_normal(N))
    ll_new[5] = -np.inf
    g_new = rng.standard_normal((N, D))
    g_new[2, 1] = np.nan
    g_new[6, 0] = np.inf
    m0, s0 = np.zeros(D), np.ones(D)
    rec = smc2.update(st, k, th_new, ll_new, g_new, 7, 0.2, "langevin", m0, s0)
    lw = rec["logw"]
    assert lw[2] == -np.inf and lw[6] == -np.inf and lw[5] == -np.inf
    live = [0, 1, 3, 4, 7]
    assert np.all(np.isfinite(lw[live]))
    assert np.all(np.isfinite(rec["mean"])) and rec["ess"] > 1.0
    w = np.exp(lw[live] - lw[live].max())
    np.testing.assert_allclose(rec["mean"], w @ th_new[live] / w.sum(), rtol=1e-12)
    # the random walk ignores the gradient
    st2 = smc2.State(N, D)
    st2.theta, st2.gradpi, st2.logpi, st2.logw = st.theta, st.gradpi, st.logpi, np.zeros(N)
    rec2 = smc2.update(st2, k, th_new, ll_new, g_new, 7, 0.2, "rw", m0, s0)
    assert np.isfinite(rec2["logw"][2]) and np.isfinite(rec2["logw"][6])


def _gauss_fn(mu_l, s_l):
    def fn(th):
        z = (th - mu_l) / s_l
        return -0.5 * np.sum(z * z, axis=-1), -z / s_l
    return fn


def test_leapfrog_is_reversible_and_nearly_conserves_energy():
    """Leapfrog steps are exactly reversible: from the end point with the momentum negated,
    the same number of steps returns to the start with the start momentum negated (an
    error in a kick or its placement breaks this); on a Gaussian target the Hamiltonian
    -log pi + |v|^2 / (2 gamma^2) changes by O(step^2) only."""
    rng = np.random.default_rng(8)
    mu_l, s_l = np.array([0.4, -0.2, 1.0]), np.array([0.5, 0.8, 0.3])
    fn = _gauss_fn(mu_l, s_l)
    grad = lambda th, l: fn(th)
    th0 = rng.standard_normal((20, 3))
    gamma = 0.05
    v0 = gamma * rng.standard_normal((20, 3))
    _, g0 = fn(th0)
    thL, vL, lpL, gL, lps = smc2.leapfrog(th0, v0, g0, 7, gamma, grad)
    assert len(lps) == 7
    thB, vB, _, _, _ = smc2.leapfrog(thL, -vL, gL, 7, gamma, grad)
    np.testing.assert_allclose(thB, th0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(vB, -v0, rtol=0, atol=1e-12)
    lp0, _ = fn(th0)
    H0 = -lp0 + 0.5 * np.sum(v0 * v0, axis=1) / gamma ** 2
    HL = -lpL + 0.5 * np.sum(vL * vL, axis=1) / gamma ** 2
    assert np.max(np.abs(HL - H0)) < 0.05 * np.max(np.abs(H0))


def test_hmc_with_one_step_is_the_langevin_move():
    """One leapfrog step is the SMC1 move (Sec. III-D) and its momentum-reversal weight is
    the Langevin L-kernel weight: the two samplers agree to rounding."""
    fn = _gauss_fn(np.array([0.8, -0.5, 0.3]), np.array([0.3, 0.4, 0.25]))
    y = np.zeros((1, 1), np.float32)
    a, _ = smc2.run(0, 1, 1, None, y, 256, 1, 8, 0.4, "langevin", 321, loglik_grad_fn=fn, D=3)
    b, _ = smc2.run(0, 1, 1, None, y, 256, 1, 8, 0.4, "hmc", 321, loglik_grad_fn=fn, D=3, hmc_steps=1)
    for ra, rb in zip(a, b):
        assert ra["resampled"] == rb["resampled"]
        np.testing.assert_allclose(rb["theta"], ra["theta"], rtol=0, atol=1e-12)
        np.testing.assert_allclose(rb["logw"], ra["logw"], rtol=0, atol=1e-9)


def test_hmc_sampler_recovers_conjugate_gaussian_posterior():
    """Three leapfrog steps per move, exact Gaussian likelihood: the recycled estimate and
    the weighted spread match the closed-form posterior (a wrong kinetic-energy term in the
    weight leaves the spread of the unadjusted dynamics)."""
    mu_l = np.array([0.8, -0.5, 0.3])
    s_l = np.array([0.3, 0.4, 0.25])
    prec = 1.0 + 1.0 / s_l ** 2
    post_mean = (mu_l / s_l ** 2) / prec
    post_var = 1.0 / prec
    N = 3000
    recs, rec_mean = smc2.run(0, 1, 1, None, np.zeros((1, 1), np.float32), N, 1, 20, 0.3, "hmc", 124,
                              loglik_grad_fn=_gauss_fn(mu_l, s_l), D=3, hmc_steps=3)
    for r in recs:
        assert 1.0 - 1e-9 <= r["ess"] <= N + 1e-9
    assert np.all(np.abs(rec_mean - post_mean) < 0.1 * np.sqrt(post_var))
    last = recs[-1]
    w = np.exp(last["logw"] - last["logw"].max())
    w /= w.sum()
    var = w @ (last["theta"] - last["mean"]) ** 2
    assert np.all((var / post_var > 0.8) & (var / post_var < 1.3)), var / post_var
