"""GPU parity of the CRN particle filter (forward + adjoint) against the FP64 oracle.

All calls go through the C ABI (libsmc2.so).  Small cases span several warps
and a ragged particle tail; the full-size cases run the whole launch of the
benchmark's configuration and check sampled filters one by one.
"""
import numpy as np
import pytest

import oracle
from paper_2407_17296_gb300 import workloads as W

from .parity import BAND, check_rows, gpu_pf

pytestmark = pytest.mark.gpu


def _report(name, agg):
    print(f"\n[{name}] " + ", ".join(f"{k}={v}" for k, v in sorted(agg.items())))


@pytest.mark.parametrize("make,T,M,n", [(W.lg1, 80, 300, 9), (W.lg4, 60, 1000, 7), (W.sv, 90, 517, 6),
                                        (W.lg16, 30, 250, 4), (W.lgssm, 80, 250, 6)])
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("kc", [1, 7])
def test_parity_small(make, T, M, n, scheme, kc):
    w = make(T=T, N=n, M=M)
    theta = W.thetas_near(w, n, 0.05, seed=11)
    ll, g, anc, flag = gpu_pf(w, theta, iteration=3, pf_resample=scheme, ckpt_every=kc)
    agg = check_rows(w, theta, ll, g, anc, flag, range(n), iteration=3, scheme=scheme,
                     name=f"small {w.name} T={T} M={M} scheme={scheme} kc={kc}")
    assert agg["resample_steps"] > 0
    _report(f"{w.name} T={T} M={M} scheme={scheme} kc={kc}", agg)


@pytest.mark.parametrize("ppt", [1, 2, 4, 8])
def test_parity_particles_per_thread(ppt):
    w = W.lg4(T=40, N=3, M=333)
    theta = W.thetas_near(w, 3, 0.05, seed=5)
    ll, g, anc, flag = gpu_pf(w, theta, particles_per_thread=ppt, ckpt_every=3)
    check_rows(w, theta, ll, g, anc, flag, range(3))


def _spread(N, ends, stride, start):
    """Rows at the ends of the launch and of its two halves, and every stride-th row between."""
    return sorted(set(ends) | set(range(start, N, stride)))


def test_parity_full_size_lg4():
    """Full linear-Gaussian workload (N=1024, M=1024, T=250) in the benchmark's launch
    configuration (two halves of 512 filters on two streams); 70 filters checked one by one,
    among them the first and last of each half."""
    w = W.lg4()
    theta = W.thetas_near(w, w.N, 0.05, seed=21)
    ll, g, anc, flag = gpu_pf(w, theta, iteration=2)
    assert np.all(np.isfinite(ll)) and np.all(np.isfinite(g))
    rows = _spread(w.N, [0, 1, 2, 255, 256, 511, 512, 513, 767, 1021, 1022, 1023], 17, 3)
    assert len(rows) >= 64
    agg = check_rows(w, theta, ll, g, anc, flag, rows, iteration=2, name="full lg4 N=1024 M=1024 T=250")
    _report("lg4 full", agg)


def test_parity_full_size_lg16():
    """Full 16-dimensional workload (N=2048, M=1024, T=200, D=48; each particle spread over
    two lanes forward and four in the adjoint); 35 filters checked one by one."""
    w = W.lg16()
    theta = W.thetas_near(w, w.N, 0.03, seed=23)
    ll, g, anc, flag = gpu_pf(w, theta, iteration=2)
    assert np.all(np.isfinite(ll)) and np.all(np.isfinite(g))
    rows = _spread(w.N, [0, 1023, 1024, 2047], 67, 7)
    assert len(rows) >= 32
    agg = check_rows(w, theta, ll, g, anc, flag, rows, iteration=2, name="full lg16 N=2048 M=1024 T=200")
    _report("lg16 full", agg)


@pytest.mark.parametrize("ppt", [4, 8])
def test_parity_lg16_particles_per_thread(ppt):
    w = W.lg16(T=20, N=2, M=500)
    theta = W.thetas_near(w, 2, 0.03, seed=6)
    ll, g, anc, flag = gpu_pf(w, theta, particles_per_thread=ppt, ckpt_every=6)
    check_rows(w, theta, ll, g, anc, flag, range(2))


def test_parity_full_size_lgssm():
    """The model of Sec. IV-A with the optimal proposal at the paper's sizes (N=64, M=250,
    T=500); every filter checked."""
    w = W.lgssm()
    theta = W.thetas_near(w, w.N, 0.05, seed=24)
    ll, g, anc, flag = gpu_pf(w, theta, iteration=2, ess_frac=0.9)
    assert np.all(np.isfinite(ll)) and np.all(np.isfinite(g))
    agg = check_rows(w, theta, ll, g, anc, flag, range(w.N), iteration=2, ess_frac=0.9,
                     name="full lgssm N=64 M=250 T=500")
    assert agg["resample_steps"] > 0
    _report("lgssm full", agg)


def test_parity_full_size_sv():
    """Full stochastic-volatility workload (N=4096, M=2048, T=500); 36 filters checked."""
    w = W.sv()
    theta = W.thetas_near(w, w.N, 0.05, seed=22)
    ll, g, anc, flag = gpu_pf(w, theta, iteration=2)
    assert np.all(np.isfinite(ll)) and np.all(np.isfinite(g))
    rows = _spread(w.N, [0, 2047, 2048, 4095], 131, 5)
    assert len(rows) >= 32
    agg = check_rows(w, theta, ll, g, anc, flag, rows, iteration=2, name="full sv N=4096 M=2048 T=500")
    _report("sv full", agg)


def test_checkpoint_interval_does_not_change_results():
    w = W.lg4(T=45, N=5, M=200)
    theta = W.thetas_near(w, 5, 0.05)
    ref = gpu_pf(w, theta, ckpt_every=1)
    for kc in (2, 4, 16, 45, 64):
        out = gpu_pf(w, theta, ckpt_every=kc)
        np.testing.assert_array_equal(out[0], ref[0])
        np.testing.assert_allclose(out[1], ref[1], rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("make", [W.lg4, W.lg1, W.lg16])
def test_deterministic_and_row_offset(make, scheme):
    """Repeated launches give bit-identical log-likelihoods and gradients, for both resamplers
    (the multinomial adjoint sums its cotangents in fixed point, independent of the order of
    its atomics); rows launched on their own with the Philox row offset give the same filters."""
    w = make(T=30, N=8, M=200 if make is not W.lg16 else 128)
    theta = W.thetas_near(w, 8, 0.05 if make is not W.lg16 else 0.03)
    a = gpu_pf(w, theta, pf_resample=scheme, ess_frac=1.0)
    for _ in range(3):
        b = gpu_pf(w, theta, pf_resample=scheme, ess_frac=1.0)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
    c = gpu_pf(w, theta[3:], row0=3, pf_resample=scheme, ess_frac=1.0)
    np.testing.assert_array_equal(c[0], a[0][3:])
    np.testing.assert_array_equal(c[1], a[1][3:])


@pytest.mark.parametrize("scheme", [0, 1])
def test_two_stream_halves_match_single_launches(scheme):
    """A launch over more filters than the GPU holds at once (1024 filters of 1024 4-d
    particles) runs as two halves on two streams; every filter's log-likelihood, gradient,
    ancestors and resampling flags equal those of launches small enough to run whole."""
    from paper_2407_17296_gb300 import binding
    w = W.lg4(T=40, N=1024, M=1024)
    theta = W.thetas_near(w, w.N, 0.05, seed=31)
    n0 = binding.kernel_launches()
    a = gpu_pf(w, theta, iteration=4, pf_resample=scheme)
    assert binding.kernel_launches() - n0 == 4  # two halves x (forward, adjoint)
    for r0 in range(0, w.N, 256):
        n0 = binding.kernel_launches()
        c = gpu_pf(w, theta[r0:r0 + 256], iteration=4, row0=r0, pf_resample=scheme)
        assert binding.kernel_launches() - n0 == 2
        for x, y in zip(c, a):
            np.testing.assert_array_equal(x, y[r0:r0 + 256])


def test_single_particle_closed_form():
    """M = 1: resampling is the identity and log p-hat is the path density."""
    w = W.lg4(T=50, N=2, M=1)
    theta = W.thetas_near(w, 2, 0.1)
    ll, g, anc, flag = gpu_pf(w, theta)
    for i in range(2):
        r = oracle.pf(0, 4, 2, w.H, theta[i], w.y, 1, w.seed, 1, i)
        assert abs(ll[i] - r["loglik"]) <= 1e-4 * abs(r["loglik"])
        np.testing.assert_allclose(g[i], r["grad"], rtol=1e-3, atol=1e-3)


def test_single_step_and_forward_only():
    w = W.lg1(T=1, N=3, M=64)
    theta = W.thetas_near(w, 3, 0.1)
    ll, g, anc, flag = gpu_pf(w, theta)
    check_rows(w, theta, ll, g, anc, flag, range(3))
    ll2, g2, _, _ = gpu_pf(w, theta, want_grad=False)
    np.testing.assert_array_equal(ll, ll2)
    assert g2 is None


@pytest.mark.parametrize("ess_frac", [0.0, 1.0])
def test_never_and_always_resample(ess_frac):
    w = W.lg4(T=30, N=3, M=256)
    theta = W.thetas_near(w, 3, 0.05)
    ll, g, anc, flag = gpu_pf(w, theta, ess_frac=ess_frac)
    if ess_frac == 0.0:
        assert flag.sum() == 0
    else:
        assert np.all(flag[:, 1:] == 1)
    check_rows(w, theta, ll, g, anc, flag, range(3), ess_frac=ess_frac)


def test_degenerate_filter_reports_minus_inf():
    """Exploding dynamics overflow FP32 for every particle: log p-hat = -inf, gradient 0,
    and the neighbouring filters of the launch are unaffected."""
    w = W.lg1(T=100, N=3, M=64)
    theta = W.thetas_near(w, 3, 0.05)
    theta[1, 0] = 40.0
    ll, g, anc, flag = gpu_pf(w, theta)
    assert ll[1] == -np.inf and np.all(g[1] == 0.0)
    check_rows(w, theta, ll, g, anc, flag, [0, 2])


def test_zero_rows_is_a_noop():
    import torch
    from paper_2407_17296_gb300 import binding
    w = W.lg1(T=10, N=4, M=32)
    with binding.Handle(binding.config_for(w)) as h:
        th = torch.zeros(0, 3, dtype=torch.float64, device="cuda")
        ll = torch.zeros(0, dtype=torch.float64, device="cuda")
        h.pf_loglik_grad(th, 1, ll, None)
        torch.cuda.synchronize()


def test_host_buffer_entry_point_matches_device():
    from paper_2407_17296_gb300 import binding
    w = W.lg4(T=25, N=6, M=100)
    theta = W.thetas_near(w, 6, 0.05)
    ll_d, g_d, _, _ = gpu_pf(w, theta)
    with binding.Handle(binding.config_for(w)) as h:
        ll = np.zeros(6)
        g = np.zeros((6, w.D))
        h.pf_loglik_grad_host(np.ascontiguousarray(theta), 1, ll, g)
    np.testing.assert_array_equal(ll, ll_d)
    np.testing.assert_array_equal(g, g_d)


def test_autograd_function():
    import torch
    from paper_2407_17296_gb300 import autograd, binding
    w = W.lg4(T=20, N=4, M=128)
    theta = W.thetas_near(w, 4, 0.05)
    ll_ref, g_ref, _, _ = gpu_pf(w, theta)
    with binding.Handle(binding.config_for(w)) as h:
        th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
        ll = autograd.loglik(th, h, 1)
        wts = torch.arange(1, 5, dtype=torch.float64, device="cuda")
        (ll * wts).sum().backward()
        np.testing.assert_array_equal(ll.detach().cpu().numpy(), ll_ref)
        np.testing.assert_allclose(th.grad.cpu().numpy(), g_ref * np.arange(1, 5)[:, None], rtol=1e-12)


def test_autograd_orders_with_a_busy_current_stream():
    """The handle runs on its own stream while torch's current stream is still producing theta
    (a long chain of kernels before the copy that writes it) and consumes the outputs right
    away: the Function's event ordering makes the results equal those of a quiet run."""
    import torch
    from paper_2407_17296_gb300 import autograd, binding
    w = W.lg4(T=20, N=4, M=128)
    theta = W.thetas_near(w, 4, 0.05)
    ll_ref, g_ref, _, _ = gpu_pf(w, theta)
    src = torch.tensor(theta, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    with binding.Handle(binding.config_for(w)) as h:
        assert h.stream_ptr() != side.cuda_stream
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            x = torch.randn(2048, 2048, device="cuda")
            for _ in range(30):  # tens of milliseconds of work ahead of theta on this stream
                x = torch.tanh(x @ x)
            th = (src + 0.0 * x[0, 0].double()).requires_grad_(True)
            ll = autograd.loglik(th, h, 1)
            out = ll * 1.0  # consumed on the current stream at once
            out.sum().backward()
            gr = th.grad.clone()
        torch.cuda.synchronize()
    np.testing.assert_array_equal(out.detach().cpu().numpy(), ll_ref)
    np.testing.assert_array_equal(gr.cpu().numpy(), g_ref)


@pytest.mark.parametrize("make,M,n", [(W.lg16, 2048, 2), (W.lg4, 4096, 2)])
def test_parity_large_blocks(make, M, n):
    """Block sizes whose adjoint cannot keep four (or two) state slices in shared memory:
    the 4-d model with M = 4096 runs a two-slot ring, the 16-d model with M = 2048 reads the
    slices from memory."""
    w = make(T=12, N=n, M=M)
    theta = W.thetas_near(w, n, 0.03, seed=31)
    for scheme in (0, 1):
        ll, g, anc, flag = gpu_pf(w, theta, pf_resample=scheme)
        check_rows(w, theta, ll, g, anc, flag, range(n), scheme=scheme)


def test_bounded_wait_reports_timeout_and_context_survives():
    """Failure detection without a fault: a wait that nothing completes gives up after its poll
    limit, the status word says so, and the filters still run afterwards."""
    from paper_2407_17296_gb300 import binding
    assert binding.selftest_bounded_wait(2000) is True
    w = W.lg1(T=10, N=2, M=64)
    theta = W.thetas_near(w, 2, 0.05)
    ll, g, anc, flag = gpu_pf(w, theta)
    assert np.all(np.isfinite(ll))
