"""The seeded synthetic workloads: sizes and parameters as stated, reproducible series,
simulators that follow the models (stationary moments of long simulated series), and the
serving stream's job mix.  CPU only."""
import numpy as np
import pytest

from paper_2407_17296_gb300 import workloads as W

SIZES = {  # name: (family, d_x, d_y, D, T, N, M)
    "lg1": (W.LG_DIAG, 1, 1, 3, 100, 64, 128),
    "lg4": (W.LG_DIAG, 4, 2, 10, 250, 1024, 1024),
    "sv": (W.SV, 1, 1, 3, 500, 4096, 2048),
    "lg16": (W.LG_DIAG, 16, 16, 48, 200, 2048, 1024),
    "lgssm": (W.LG_OPT, 1, 1, 3, 500, 64, 250),
}


@pytest.mark.parametrize("name", sorted(SIZES))
def test_sizes_and_reproducible_series(name):
    w = W.ALL[name]()
    fam, dx, dy, D, T, N, M = SIZES[name]
    assert (w.family, w.dx, w.dy, w.D, w.T, w.N, w.M) == (fam, dx, dy, D, T, N, M)
    assert w.theta_star.shape == (D,)
    assert w.y.shape == (T, dy) and w.y.dtype == np.float32 and np.all(np.isfinite(w.y))
    if w.H is not None:
        assert w.H.shape == (dy, dx)
    np.testing.assert_array_equal(W.ALL[name]().y, w.y)  # same data seed, same series
    short = w.with_sizes(T=T // 2)
    np.testing.assert_array_equal(short.y, w.y[:T // 2])
    with pytest.raises(ValueError):
        w.with_sizes(T=T + 1)


def test_step_sizes_scale_with_the_series_length():
    s = W.step_sizes(500)
    assert (s["langevin"], s["rw"], s["hmc"]) == (0.085, 0.175, 0.085)
    assert W.step_sizes(125)["langevin"] == pytest.approx(0.17)
    assert W.lg1().gamma == pytest.approx(0.085 * np.sqrt(5.0))


def test_lg1_series_has_the_stationary_variance():
    """y_t = x_t + w_t with x_t stationary AR(1): var y = q^2 / (1 - a^2) + r^2
    (a = 0.8, q = 0.5, r = 1: 1.694) and lag-1 autocovariance a q^2 / (1 - a^2)."""
    y = W.lg1(T=200000).y[1000:, 0].astype(np.float64)
    vx = 0.25 / (1 - 0.64)
    assert np.var(y) == pytest.approx(vx + 1.0, rel=0.03)
    c1 = np.mean((y[1:] - y.mean()) * (y[:-1] - y.mean()))
    assert c1 == pytest.approx(0.8 * vx, rel=0.06)


def test_sv_series_has_the_stationary_second_moment():
    """y_t = exp(x_t / 2) e_t with x_t ~ N(mu, sigma^2 / (1 - phi^2)) stationary:
    E y^2 = exp(mu + sigma^2 / (2 (1 - phi^2)))."""
    y = W.sv(T=400000).y[:, 0].astype(np.float64)
    mu, phi, sig = -1.0, 0.95, 0.25
    want = np.exp(mu + sig * sig / (2 * (1 - phi * phi)))
    assert np.mean(y * y) == pytest.approx(want, rel=0.06)


def test_lg4_observation_matrix_and_dynamics():
    w = W.lg4()
    a = w.theta_star[:4]
    assert np.all((a >= 0) & (a < 0.95))
    np.testing.assert_allclose(w.theta_star[4:8], np.log(0.5))
    np.testing.assert_allclose(w.theta_star[8:], 0.0)
    # H ~ N(0, 1) / 2 entry-wise: an 8-entry sample, loosely
    assert 0.05 < np.std(w.H) < 1.5


def test_thetas_near_is_seeded_and_centred():
    w = W.lg4()
    a = W.thetas_near(w, 4096, 0.05, seed=1)
    np.testing.assert_array_equal(a, W.thetas_near(w, 4096, 0.05, seed=1))
    np.testing.assert_allclose(a.mean(axis=0), w.theta_star, atol=0.01)
    np.testing.assert_allclose(a.std(axis=0), 0.05, rtol=0.1)


def test_serving_stream_job_mix():
    jobs = W.serving_stream()
    assert len(jobs) == 256
    t = np.array([tj for tj, _ in jobs])
    assert np.all(np.diff(t) > 0)
    names, Ns, Ms = set(), set(), set()
    for _, w in jobs:
        assert 50 <= w.T <= 1000 and w.y.shape == (w.T, w.dy)
        names.add(w.name)
        Ns.add(w.N)
        Ms.add(w.M)
        assert w.gamma == pytest.approx(W.step_sizes(w.T)["langevin"])
    assert names == {"lg1", "lg4", "sv", "lg16"}
    assert Ns == {256, 1024, 4096} and Ms == {128, 512, 2048}
    # Poisson arrivals at 50 jobs/s: mean gap 20 ms
    assert np.mean(np.diff(t)) == pytest.approx(0.02, rel=0.2)
    # each job has its own seed and series
    assert len({w.seed for _, w in jobs}) == 256
