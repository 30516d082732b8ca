"""The split SMC^2 step (smc2_step_filters / smc2_step_update) on the GPU.

Two handles stand for two ranks: each filters its own block of rows, the blocks are
concatenated (the all-gather of a real run), and both complete the iteration.  Both
replicas must equal, bit for bit, one handle running smc2_step.  A world-size-1 NCCL group
drives the same path through paper_2407_17296_gb300.sharded."""
import numpy as np
import pytest
import torch

from paper_2407_17296_gb300 import binding, workloads
from paper_2407_17296_gb300.sharded import shard_rows

pytestmark = pytest.mark.gpu


def _ref_run(w, K):
    with binding.Handle(binding.config_for(w)) as h:
        stats = [h.step() for _ in range(K)]
        th, lw = h.samples()
    return stats, th, lw


# 1024 filters of 1024 particles exceed one forward wave: the single handle's steps (a
# replayed graph) run them as two halves on two streams, each replica's 512 rows as one
# launch per pass, so the comparison also pins the halves to the single launch
@pytest.mark.parametrize("N,M", [(10, 256), (9, 256), (1024, 1024)])
def test_two_replicas_equal_one_handle(N, M):
    w = workloads.lg4(T=30, N=N, M=M, K=3)
    K = 3
    stats_ref, th_ref, lw_ref = _ref_run(w, K)
    dev = torch.device("cuda")
    hs = [binding.Handle(binding.config_for(w)) for _ in range(2)]
    try:
        for k in range(K):
            lls, gs = [], []
            for r, h in enumerate(hs):
                row0, n = shard_rows(N, 2, r)
                ll = torch.empty(n, dtype=torch.float64, device=dev)
                g = torch.empty(n, w.D, dtype=torch.float64, device=dev)
                h.step_filters(row0, n, ll, g)
                lls.append(ll)
                gs.append(g)
            torch.cuda.synchronize()
            ll_all, g_all = torch.cat(lls), torch.cat(gs)
            for h in hs:
                st = h.step_update(ll_all, g_all)
                assert st["k"] == stats_ref[k]["k"]
                assert st["ess"] == stats_ref[k]["ess"]
                assert st["resampled"] == stats_ref[k]["resampled"]
                np.testing.assert_array_equal(st["mean"], stats_ref[k]["mean"])
        for h in hs:
            th, lw = h.samples()
            np.testing.assert_array_equal(th, th_ref)
            np.testing.assert_array_equal(lw, lw_ref)
    finally:
        for h in hs:
            h.close()


def test_split_calls_must_alternate():
    w = workloads.lg1(T=10, N=4, M=32)
    dev = torch.device("cuda")
    with binding.Handle(binding.config_for(w)) as h:
        ll = torch.empty(4, dtype=torch.float64, device=dev)
        g = torch.empty(4, w.D, dtype=torch.float64, device=dev)
        with pytest.raises(binding.Smc2Error):
            h.step_update(ll, g)
        with pytest.raises(binding.Smc2Error):
            h.step_filters(3, 2, ll, g)  # rows beyond N
        h.step_filters(0, 4, ll, g)
        with pytest.raises(binding.Smc2Error):
            h.step_filters(0, 4, ll, g)
        h.step_update(ll, g)


def test_sharded_driver_nccl_world_one():
    import socket
    import torch.distributed as dist
    from paper_2407_17296_gb300 import sharded
    w = workloads.lg4(T=25, N=8, M=128, K=2)
    stats_ref, th_ref, _ = _ref_run(w, 2)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    try:
        stream = torch.cuda.Stream()
        with binding.Handle(binding.config_for(w, stream=stream.cuda_stream)) as h:
            drv = sharded.ShardedSMC2(sharded.HandleEngine(h, stream), w.N, w.D)
            for k in range(2):
                st = drv.step()
                assert st["ess"] == stats_ref[k]["ess"]
            th, _ = h.samples()
            np.testing.assert_array_equal(th, th_ref)
    finally:
        dist.destroy_process_group()


def test_two_processes_cuda_engine_gloo_exchange():
    """Two processes, each a rank with its own handle on the same GPU (their kernels never wait
    on one another), filter their halves of the rows; the rows are exchanged by a gloo
    all-gather through host memory.  Both replicas equal one handle running smc2_step."""
    import multiprocessing as mp
    import socket
    from .sharded_cuda_worker import worker
    N, K = 24, 3
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=worker, args=(r, 2, port, N, K, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(2)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in res:
        assert r[1] >= 0, r[5]
    assert [(r[1], r[2]) for r in res] == [shard_rows(N, 2, 0), shard_rows(N, 2, 1)]
    w = workloads.lg4(T=30, N=N, M=256, K=K)
    stats_ref, th_ref, lw_ref = _ref_run(w, K)
    for r in res:
        np.testing.assert_array_equal(r[3], th_ref)
        np.testing.assert_array_equal(r[4], lw_ref)
        assert [s[1] for s in r[5]] == [st["ess"] for st in stats_ref]
        assert [s[2] for s in r[5]] == [st["resampled"] for st in stats_ref]
