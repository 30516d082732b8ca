"""An engine for paper_2407_17296_gb300.sharded built from the oracle (CPU, FP64), so the
row partition and the exchange of the sharded sampler can be tested on gloo ranks."""
import numpy as np
import torch

from oracle import smc2 as osmc2


class OracleEngine:
    def __init__(self, w, N):
        self.w = w
        self.N, self.D = N, w.D
        self.m0 = np.zeros(w.D) if w.prior_mean is None else np.asarray(w.prior_mean, dtype=np.float64)
        self.s0 = np.ones(w.D) if w.prior_std is None else np.asarray(w.prior_std, dtype=np.float64)
        self.state = osmc2.State(N, w.D)
        self.k = 0
        self.theta_new = None
        self.device = torch.device("cpu")

    def step_filters(self, row0, n):
        w = self.w
        self.theta_new = osmc2.propose(self.state, self.k + 1, w.seed, w.gamma, w.proposal, self.m0, self.s0)
        ll, g, _, _ = osmc2.run_filters(w.family, w.dx, w.dy, w.H, w.y, w.M, w.seed, self.k + 1,
                                        self.theta_new, range(row0, row0 + n))
        return torch.from_numpy(ll), torch.from_numpy(g)

    def step_update(self, ll_all, g_all):
        w = self.w
        self.k += 1
        rec = osmc2.update(self.state, self.k, self.theta_new, ll_all.numpy().copy(), g_all.numpy().copy(),
                           w.seed, w.gamma, w.proposal, self.m0, self.s0)
        return {"k": rec["k"], "ess": rec["ess"], "l_k": rec["l_k"], "resampled": rec["resampled"],
                "mean": rec["mean"]}


def worker(rank, world, port, N, K, out_q):
    """One gloo rank: K sharded iterations of the small 1-D workload; sends its final state."""
    import torch.distributed as dist
    from paper_2407_17296_gb300 import sharded, workloads
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w = workloads.lg1(T=12, N=N, M=32, K=K)
        eng = OracleEngine(w, N)
        drv = sharded.ShardedSMC2(eng, N, w.D)
        stats = [drv.step() for _ in range(K)]
        out_q.put((rank, drv.row0, drv.n, eng.state.theta, eng.state.logw, eng.state.loglik,
                   [(s["k"], s["ess"], s["resampled"]) for s in stats]))
    finally:
        dist.destroy_process_group()
