"""Continuous-batching server: jobs of different model families and sizes submitted
together overlap on the GPU, and each job's result is the same as when it runs alone
(every kernel is deterministic and each job has its own stream and state)."""
import time

import numpy as np
import pytest

from paper_2407_17296_gb300 import workloads as W

pytestmark = pytest.mark.gpu


# jobs whose filters resample with the multinomial scheme (the paper's, Sec. II-B)
MULTINOMIAL_JOBS = (7, 8)


def _jobs():
    from dataclasses import replace
    return [W.lg1(T=50, N=64, M=128, K=3), W.lg4(T=40, N=32, M=256, K=3),
            W.sv(T=60, N=48, M=128, K=4), W.lg16(T=20, N=16, M=128, K=2),
            W.lg4(T=30, N=64, M=100, K=2, proposal="rw"),
            replace(W.lg1(T=50, N=64, M=128, K=3, proposal="hmc"), hmc_steps=2, gamma=0.1),
            replace(W.lg1(T=40, N=32, M=128, K=3, proposal="nuts"), nuts_depth=2, gamma=0.1),
            W.lg4(T=40, N=32, M=256, K=3), W.sv(T=60, N=48, M=128, K=3)]


def _cfg(i, w):
    from paper_2407_17296_gb300 import binding
    return binding.config_for(w, pf_resample=1 if i in MULTINOMIAL_JOBS else 0)


def _alone(i, w):
    from paper_2407_17296_gb300 import binding
    with binding.Handle(_cfg(i, w)) as h:
        st = None
        for _ in range(w.K):
            st = h.step()
        th, lw = h.samples()
    return th, lw, st["recycled_mean"]


def _wait(server, ids, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(ids):
        for j in ids:
            if j not in out:
                r = server.poll(j)
                if r is not None:
                    out[j] = r
        assert time.time() - t0 < timeout, "served jobs did not finish"
        time.sleep(0.002)
    return out


@pytest.mark.parametrize("fused", [True, False])
def test_results_alone_equal_results_in_the_mix(fused):
    """With fused batching (ready jobs step together, filter passes of jobs of one kernel variant
    in one persistent launch) and without it (one stream a job)."""
    from paper_2407_17296_gb300 import binding
    jobs = _jobs()
    alone = [_alone(i, w) for i, w in enumerate(jobs)]
    with binding.Server(hbm_budget=8 << 30, max_active=8) as srv:
        srv.set_fused(fused)
        ids = [srv.submit(_cfg(i, w)) for i, w in enumerate(jobs)]
        res = _wait(srv, ids)
    for w, j, (th, lw, rec) in zip(jobs, ids, alone):
        r = res[j]
        assert r["status"] == 0 and r["K"] == w.K
        np.testing.assert_array_equal(r["theta"], th)
        np.testing.assert_array_equal(r["logw"], lw)
        np.testing.assert_array_equal(r["recycled_mean"], rec)
        assert r["latency_s"] >= r["queue_s"] >= 0.0


def test_admission_by_footprint_and_rejection():
    """Admission by footprint: a job that fixes its checkpoint interval waits until memory frees
    up; a job with the automatic interval is admitted at once with a longer interval (fewer
    stored steps) when that fits the room left; a job that cannot fit even then is rejected."""
    from paper_2407_17296_gb300 import binding
    small = W.lg4(T=40, N=32, M=256, K=2)
    fp = binding.footprint(binding.config_for(small))  # the automatic interval stores every step
    fp_min = min(binding.footprint(binding.config_for(small, ckpt_every=k)) for k in (2, 4, 8, 16, 32))
    assert fp_min < 0.5 * fp
    # room for one job at a time: the second waits until the first frees its memory
    with binding.Server(hbm_budget=int(fp * 1.5), max_active=8) as srv:
        ids = [srv.submit(binding.config_for(small, ckpt_every=1)) for _ in range(3)]
        res = _wait(srv, ids)
        assert all(res[j]["status"] == 0 for j in ids)
        first, second = res[ids[0]], res[ids[1]]
        assert second["queue_s"] >= 0.5 * (first["latency_s"] - first["queue_s"])
        big = binding.config_for(W.lg4(T=40, N=1024, M=1024, K=1))
        with pytest.raises(binding.Smc2Error, match="NOMEM"):
            srv.submit(big)
    # room for one job and a bit: the second is admitted next to the first, with a longer interval
    with binding.Server(hbm_budget=int(fp + 1.05 * fp_min), max_active=8) as srv:
        ids = [srv.submit(binding.config_for(small)) for _ in range(2)]
        res = _wait(srv, ids)
        assert all(res[j]["status"] == 0 for j in ids)
        first, second = res[ids[0]], res[ids[1]]
        assert second["queue_s"] < first["latency_s"] - first["queue_s"]


def test_cancel_and_unknown_ids():
    from paper_2407_17296_gb300 import binding
    w = W.lg4(T=40, N=32, M=256, K=50)
    with binding.Server(hbm_budget=1 << 30, max_active=1) as srv:
        a = srv.submit(binding.config_for(w))
        b = srv.submit(binding.config_for(w))
        srv.cancel(b)  # still queued behind a
        with pytest.raises(binding.Smc2Error, match="NOTFOUND"):
            srv.poll(b)
        srv.cancel(a)
        with pytest.raises(binding.Smc2Error):
            srv.poll(12345)
