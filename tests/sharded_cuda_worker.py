"""A rank of the sharded SMC^2 sampler with the CUDA engine (binding.Handle) on cuda:0 and a
gloo process group: the filter outputs travel through host memory in the all-gather.  Run as a
spawned process by tests/test_gpu_sharded.py; puts (rank, row0, n, theta, logw, stats) on q."""


def worker(rank, world, port, N, K, q):
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from paper_2407_17296_gb300 import binding, sharded, workloads
    try:
        dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
        torch.cuda.set_device(0)
        w = workloads.lg4(T=30, N=N, M=256, K=K)
        stream = torch.cuda.Stream()
        with binding.Handle(binding.config_for(w, stream=stream.cuda_stream)) as h:
            drv = sharded.ShardedSMC2(sharded.HandleEngine(h, stream), w.N, w.D, device=torch.device("cpu"))
            stats = []
            for _ in range(K):
                st = drv.step()
                stats.append((st["k"], st["ess"], st["resampled"]))
            th, lw = h.samples()
        q.put((rank, drv.row0, drv.n, th, lw, stats))
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, -1, -1, None, None, repr(e)))
