"""Fused iterations of several jobs (smc2_batch_step): the filter passes of jobs that share a
kernel variant run as one persistent multi-job launch, and every job's result is bit-identical
to the same job stepped on its own (the filters of an iteration are independent, Table I)."""
import numpy as np
import pytest

from paper_2407_17296_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _jobs():
    from dataclasses import replace
    return [  # (workload, extra config)
        (W.lg4(T=40, N=40, M=256, K=3), {}),
        (W.lg4(T=25, N=16, M=256, K=3, proposal="rw"), {"pf_resample": 1}),
        (replace(W.lg4(T=33, N=7, M=256, K=3), seed=4242), {"ess_frac": 0.9}),
        (W.lg4(T=30, N=12, M=250, K=3), {}),           # another M, the same block size
        (W.lg1(T=50, N=64, M=128, K=3), {}),
        (replace(W.lg1(T=20, N=30, M=128, K=3), seed=99), {}),
        (W.sv(T=40, N=24, M=128, K=3), {}),
        (replace(W.lg1(T=30, N=32, M=128, K=3, proposal="hmc"), hmc_steps=2, gamma=0.1), {}),
        (replace(W.lg1(T=30, N=24, M=128, K=3, proposal="nuts"), nuts_depth=2, gamma=0.1), {}),
        (W.lgssm(T=60, N=32, M=250, K=3), {}),         # optimal proposal, uniform priors
        (replace(W.lgssm(T=45, N=20, M=250, K=3, proposal="rw"), seed=31), {}),
    ]


def _alone(w, kw):
    from paper_2407_17296_gb300 import binding
    out = []
    with binding.Handle(binding.config_for(w, **kw)) as h:
        for _ in range(w.K):
            st = h.step()
            out.append((st, h.samples()))
    return out


def test_batch_step_equals_each_job_alone():
    from paper_2407_17296_gb300 import binding
    jobs = _jobs()
    ref = [_alone(w, kw) for w, kw in jobs]
    hs = [binding.Handle(binding.config_for(w, **kw)) for w, kw in jobs]
    try:
        with binding.Batch(len(hs)) as b:
            for k in range(3):
                n0 = binding.kernel_launches()
                stats = b.step(hs)
                # proposal + update of every job; one fused forward and adjoint launch per group of
                # several jobs (lg4 at 128 threads, lg1, lgssm); sv alone in its group and the HMC
                # and NUTS jobs after their first iteration step on their own
                assert binding.kernel_launches() - n0 >= 5 * (len(hs) - 2) + 2 * 3
                for i, h in enumerate(hs):
                    st_ref, (th_ref, lw_ref) = ref[i][k]
                    th, lw = h.samples()
                    np.testing.assert_array_equal(th, th_ref, err_msg=f"job {i} iteration {k}")
                    np.testing.assert_array_equal(lw, lw_ref, err_msg=f"job {i} iteration {k}")
                    for key in ("k", "resampled", "ess", "l_k", "pf_near_ties", "pf_resample_steps"):
                        assert stats[i][key] == st_ref[key], (i, k, key)
                    np.testing.assert_array_equal(stats[i]["mean"], st_ref["mean"])
    finally:
        for h in hs:
            h.close()


def test_batch_of_identical_shapes_is_one_fused_pass():
    """Sixteen replicate runs of the small linear-Gaussian job (N=64, M=128: 64 filter blocks
    each, too few to fill the GPU alone) fuse into one forward and one adjoint launch."""
    from dataclasses import replace
    from paper_2407_17296_gb300 import binding
    ws = [replace(W.lg1(K=2), seed=1000 + r) for r in range(16)]
    hs = [binding.Handle(binding.config_for(w)) for w in ws]
    try:
        with binding.Batch(16) as b:
            b.step(hs)
            n0 = binding.kernel_launches()
            stats = b.step(hs)
            assert binding.kernel_launches() - n0 == 16 * 5 + 2
        for w, h, st in zip(ws, hs, stats):
            ref = _alone(w, {})
            np.testing.assert_array_equal(h.samples()[0], ref[1][1][0])
            assert st["ess"] == ref[1][0]["ess"]
    finally:
        for h in hs:
            h.close()


def test_batch_rejects_bad_arguments():
    from paper_2407_17296_gb300 import binding
    w = W.lg1(T=10, N=8, M=32, K=1)
    with binding.Handle(binding.config_for(w)) as h, binding.Batch(2) as b:
        with pytest.raises(binding.Smc2Error):
            b.step([h, h])
        with pytest.raises(binding.Smc2Error):
            b.step([h, h, h])
        assert b.step([]) == []
