"""The allocation-free entry point pf_loglik_grad_static, called through the C ABI.

For callers that cannot allocate device memory (a framework that owns all device
memory through its own pool, a latency-critical loop where cudaMalloc would
synchronise the device, a plug-in that must not grow its footprint): the filter's
working memory comes from a fixed array inside the library.  Its results must equal
those of the ordinary entry point pf_loglik_grad, on two calls in a row (the second
call reuses the array the first one left behind).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2407_17296_gb300 import workloads as W

from .parity import GRAD_RTOL, LL_RTOL, check_rows

pytestmark = pytest.mark.gpu


def _reference(w, theta, iteration):
    """The allocating entry point pf_loglik_grad on a handle: outputs and its decision trace."""
    import torch
    from paper_2407_17296_gb300 import binding
    with binding.Handle(binding.config_for(w, ckpt_every=4)) as h:
        th = torch.tensor(theta, dtype=torch.float64, device="cuda")
        ll = torch.empty(len(theta), dtype=torch.float64, device="cuda")
        g = torch.empty(len(theta), w.D, dtype=torch.float64, device="cuda")
        h.pf_loglik_grad(th, iteration, ll, g)
        torch.cuda.synchronize()
        anc, flag, _, _ = h.trace()
    return ll.cpu().numpy(), g.cpu().numpy(), anc, flag


def _static_call(lib, cfg, theta, iteration):
    import torch
    from paper_2407_17296_gb300 import binding
    th = torch.tensor(theta, dtype=torch.float64, device="cuda")
    ll = torch.empty(len(theta), dtype=torch.float64, device="cuda")
    g = torch.empty(len(theta), theta.shape[1], dtype=torch.float64, device="cuda")
    rc = lib.pf_loglik_grad_static(ctypes.byref(cfg), binding._ptr(th), len(theta), iteration, 0,
                                   binding._ptr(ll), binding._ptr(g))
    binding.check(rc, "pf_loglik_grad_static")
    torch.cuda.synchronize()
    return ll.cpu().numpy(), g.cpu().numpy()


def _assert_close(a, b):
    ll, g = a
    ll_ref, g_ref = b[:2]
    assert np.all(np.abs(ll - ll_ref) <= LL_RTOL * np.maximum(1.0, np.abs(ll_ref)))
    for i in range(len(ll)):
        gmax = max(1.0, float(np.abs(g_ref[i]).max()))
        assert float(np.abs(g[i] - g_ref[i]).max()) <= GRAD_RTOL * gmax


@pytest.mark.parametrize("make", [W.lg4, W.sv])
def test_static_entry_matches_allocating_entry_twice(make):
    import torch
    from paper_2407_17296_gb300 import binding
    lib = binding.load()
    w = make(T=60, N=6, M=256)
    y_dev = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    cfg = binding.config_for(w, ckpt_every=4)
    cfg.y = y_dev.data_ptr()
    cfg.y_on_device = 1
    # two calls in a row with different inputs: the second sees the first call's leftovers
    theta1 = W.thetas_near(w, w.N, 0.05, seed=1)
    theta2 = W.thetas_near(w, w.N, 0.05, seed=2)
    out1 = _static_call(lib, cfg, theta1, 1)
    out2 = _static_call(lib, cfg, theta2, 2)
    # no bounded wait gave up inside the calls' kernels
    assert binding.static_status() == 0
    ref1, ref2 = _reference(w, theta1, 1), _reference(w, theta2, 2)
    _assert_close(out1, ref1)
    _assert_close(out2, ref2)
    # same kernels, same launch, same inputs: identical outputs
    np.testing.assert_array_equal(out1[0], ref1[0])
    np.testing.assert_array_equal(out2[1], ref2[1])
    # and against the FP64 oracle, following the allocating run's decisions at near-ties (the
    # two entry points run the same kernels, so their decisions agree where their outputs do)
    for (ll, g), (_, _, anc, flag), theta, it in ((out1, ref1, theta1, 1), (out2, ref2, theta2, 2)):
        check_rows(w, theta, ll, g, anc, flag, range(w.N), iteration=it)


def test_static_entry_rejects_oversized_problems():
    import torch
    from paper_2407_17296_gb300 import binding
    lib = binding.load()
    w = W.lg4()  # N = 1024, M = 1024, T = 250: far beyond the fixed array
    y_dev = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    cfg = binding.config_for(w, ckpt_every=1)
    cfg.y = y_dev.data_ptr()
    cfg.y_on_device = 1
    th = torch.zeros(w.N, w.D, dtype=torch.float64, device="cuda")
    ll = torch.zeros(w.N, dtype=torch.float64, device="cuda")
    rc = lib.pf_loglik_grad_static(ctypes.byref(cfg), binding._ptr(th), w.N, 1, 0, binding._ptr(ll), None)
    assert rc == -1  # SMC2_E_INVAL
    assert "static array holds" in binding.last_error()


def test_static_entry_ignores_config_N():
    """cfg->N plays no part in the allocation-free call: N = 0 or N above the handle limit
    is accepted, the size checks use the call's n."""
    import torch
    from paper_2407_17296_gb300 import binding
    lib = binding.load()
    w = W.lg1(T=20, N=3, M=64)
    y_dev = torch.tensor(w.y, dtype=torch.float32, device="cuda")
    theta = W.thetas_near(w, 3, 0.05, seed=4)
    outs = []
    for N in (0, 3, 100000):
        cfg = binding.config_for(w, ckpt_every=2)
        cfg.N = N
        cfg.y = y_dev.data_ptr()
        cfg.y_on_device = 1
        outs.append(_static_call(lib, cfg, theta, 1))
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        np.testing.assert_array_equal(o[1], outs[0][1])
    assert binding.static_status() == 0
