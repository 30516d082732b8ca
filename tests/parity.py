"""Shared helpers of the GPU parity tests: run the CUDA path, compare with the oracle.

Tolerances (stated once, used everywhere):
  * ancestor indices and resample decisions: bit-exact, except where a
    cumulative weight lies within BAND = 1e-6 of a threshold (near-ties); the
    oracle then follows the GPU's choice and counts the case;
  * log-likelihood: |ll_gpu - ll_cpu| <= 1e-4 * max(1, |ll_cpu|);
  * gradient: max_d |g_gpu - g_cpu| <= 1e-3 * max(1, max_d |g_cpu|);
  * posterior means: |m_gpu - m_cpu| <= 1e-3 * max(1, |m_cpu|).
"""
import multiprocessing as mp
import os
from collections import Counter

import numpy as np

import oracle

BAND = 1e-6
# FP32 conditioning of the weights: where the log-weight increments accumulated since the
# last resampling reach L in magnitude, FP32 log-weights carry an absolute error of order
# 2^-24 L; the widened band max(BAND, 2^-21 L) is used for prior draws and other extreme
# parameters (counted separately as "tie_conditioned").
BAND_REL = 2.0 ** -21
LL_RTOL = 1e-4
GRAD_RTOL = 1e-3
MEAN_RTOL = 1e-3


def gpu_pf(w, theta, iteration=1, row0=0, want_grad=True, **cfgkw):
    """Run pf_loglik_grad through the C ABI; returns (ll, grad, anc, flag) as numpy."""
    import torch
    from paper_2407_17296_gb300 import binding
    cfg = binding.config_for(w, **cfgkw)
    n = theta.shape[0]
    with binding.Handle(cfg) as h:
        th = torch.tensor(theta, dtype=torch.float64, device="cuda")
        ll = torch.empty(n, dtype=torch.float64, device="cuda")
        g = torch.empty(n, w.D, dtype=torch.float64, device="cuda") if want_grad else None
        h.pf_loglik_grad(th, iteration, ll, g, row0=row0)
        torch.cuda.synchronize()
        anc, flag, _, _ = h.trace()
    return (ll.cpu().numpy(), None if g is None else g.cpu().numpy(), anc[:n], flag[:n])


# near-tie counts of every check_rows call with a name, written at the end of the session
# (conftest.py) so that a record of them exists beside the pass/fail result
TIE_REPORT = {}


def _oracle_row(args):
    (family, dx, dy, H, th, y, M, seed, iteration, row, scheme, ess_frac, want_grad, anc, flag,
     band) = args
    return oracle.pf(family, dx, dy, H, th, y, M, seed, iteration, row, scheme=scheme,
                     ess_frac=ess_frac, want_grad=want_grad, hint_anc=anc, hint_flag=flag,
                     band=band, flag_band=band)


def oracle_rows(w, theta, anc, flag, rows, iteration, row0, scheme, ess_frac, want_grad, band,
                procs=0):
    """The oracle's follow-mode run of each row; with procs > 1 in a spawn pool (safe after the
    CUDA context exists, unlike a forked one)."""
    jobs = [(w.family, w.dx, w.dy, w.H, theta[i], w.y, w.M, w.seed, iteration, row0 + i, scheme,
             ess_frac, want_grad, anc[i], flag[i], band) for i in rows]
    if procs > 1 and len(jobs) > 1:
        with mp.get_context("spawn").Pool(min(procs, len(jobs))) as pool:
            return pool.map(_oracle_row, jobs, chunksize=1)
    return [_oracle_row(j) for j in jobs]


def expected_near_ties(agg, M):
    """Thresholds within BAND of a cumulative weight occur with probability about 2 BAND M each
    (App. B's index is decided by comparisons with M cumulative weights spread over [0, 1])."""
    return 2.0 * BAND * M * M * agg["resample_steps"]


def check_rows(w, theta, ll, g, anc, flag, rows, iteration=1, row0=0, scheme=0, ess_frac=0.5,
               band=BAND, name=None, procs=0):
    """Oracle in follow mode for each sampled row; asserts the tolerances; returns counters
    (near_ties: thresholds within the band; tie_followed: of those, where the GPU chose the
    other admissible index; nontie_mismatch: a different choice outside the band, asserted 0).
    With a name the counters go into TIE_REPORT and the near-tie count is checked against its
    expected rate once 50 are expected: at most 4 times it, and at least a tenth of it (weights
    far below 1e-6 bunch their cumulative sums, which then count once)."""
    agg = Counter()
    rows = list(rows)
    res = oracle_rows(w, theta, anc, flag, rows, iteration, row0, scheme, ess_frac, g is not None,
                      band, procs=procs if procs else (os.cpu_count() or 1) if len(rows) >= 16 else 0)
    for i, r in zip(rows, res):
        st = r["stats"]
        agg.update(st)
        assert st["nontie_mismatch"] == 0, (i, st, r["worst"])
        assert st["flag_mismatch"] == 0, (i, st)
        assert st["bad_hint"] == 0, (i, st)
        np.testing.assert_array_equal(r["flag"], flag[i])
        fl = flag[i] == 1
        np.testing.assert_array_equal(r["anc"][fl], anc[i][fl])
        ref = r["loglik"]
        assert abs(ll[i] - ref) <= LL_RTOL * max(1.0, abs(ref)), (i, ll[i], ref)
        if g is not None:
            gmax = max(1.0, float(np.abs(r["grad"]).max()))
            err = float(np.abs(g[i] - r["grad"]).max())
            assert err <= GRAD_RTOL * gmax, (i, g[i], r["grad"], err / gmax)
            agg["grad_rel_err_max_e9"] = max(agg["grad_rel_err_max_e9"], int(1e9 * err / gmax))
        agg["ll_abs_err_max_e9"] = max(agg["ll_abs_err_max_e9"], int(1e9 * abs(ll[i] - ref)))
    agg["rows"] = len(rows)
    assert agg["tie_followed"] <= agg["near_ties"], agg
    if name is not None:
        exp = expected_near_ties(agg, w.M)
        if exp >= 50:
            assert exp / 10 <= agg["near_ties"] <= 4 * exp, (name, agg["near_ties"], exp)
        TIE_REPORT[name] = {**{k: int(v) for k, v in agg.items()}, "M": int(w.M), "T": int(w.T),
                            "expected_near_ties": exp,
                            "decisions": int(agg["resample_steps"]) * int(w.M)}
    return agg
