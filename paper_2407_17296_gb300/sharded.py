"""One SMC^2 job whose N particle filters are split over the ranks of a process group.

The N filters of an iteration are independent (Sec. III; the importance-sampling and
gradient rows of Table I scale as N/P), while the outer update -- L-kernel weights,
normalisation, estimate, recycling statistic, ESS, resampling (Secs. III-A..E) -- couples
all N samples but costs only O(N D).  So every rank keeps a replica of the outer state
(theta, log w, log pi-hat, grad log pi: N x (2D + 3) FP64 values) and per iteration:

  1. proposes theta' for all N samples (same Philox keys on every rank, same result) and
     runs the particle filters of its own contiguous block of rows [row0, row0 + n) with
     the Philox keys of those rows;
  2. exchanges the filter outputs (log p-hat and its gradient, 1 + D FP64 values a row)
     in ONE all-gather;
  3. applies the outer update to all N rows.

The replicas therefore stay identical, and equal to one device running every filter: the
paper's O(log2 N) redistribution between MPI ranks is replaced by one all-gather of
N (1 + D) values.  The engine does the computing (the CUDA library through
``binding.Handle``); this module only partitions rows and moves them.
"""
import torch
import torch.distributed as dist


def shard_rows(N: int, world: int, rank: int):
    """Contiguous block of rows of `rank`: (row0, n); sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, rem = divmod(N, world)
    n = base + (1 if rank < rem else 0)
    row0 = rank * base + min(rank, rem)
    return row0, n


class HandleEngine:
    """The CUDA engine: a binding.Handle whose kernels run on `stream` (a torch stream the
    handle's config was created with)."""

    def __init__(self, handle, stream):
        self.h = handle
        self.stream = stream
        self.device = stream.device
        self.D = handle.D

    def step_filters(self, row0, n):
        ll = torch.empty(n, dtype=torch.float64, device=self.device)
        g = torch.empty(n, self.D, dtype=torch.float64, device=self.device)
        self.h.step_filters(row0, n, ll, g)
        return ll, g

    def step_update(self, ll_all, g_all):
        return self.h.step_update(ll_all, g_all)


class ShardedSMC2:
    """Drive an engine (``step_filters(row0, n) -> (loglik [n], grad [n][D])`` and
    ``step_update(loglik [N], grad [N][D]) -> stats``) on every rank of `group`."""

    def __init__(self, engine, N: int, D: int, group=None, device=None):
        """device: where the exchange buffers live -- the engine's device for NCCL (default),
        the CPU for a gloo group (the rows then travel through host memory and are copied back
        to the engine's device before the update)."""
        self.engine = engine
        self.N, self.D = N, D
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.rows = [shard_rows(N, self.world, r) for r in range(self.world)]
        self.row0, self.n = self.rows[self.rank]
        self.nmax = max(n for _, n in self.rows)
        self.engine_device = getattr(engine, "device", torch.device("cpu"))
        self.device = device if device is not None else self.engine_device
        self.stream = getattr(engine, "stream", None)

    def _exchange(self, ll, g):
        # pack [n][1 + D] rows into a block padded to nmax rows, all-gather, unpack in rank order
        buf = torch.zeros(self.nmax, 1 + self.D, dtype=torch.float64, device=self.device)
        buf[:self.n, 0] = ll
        buf[:self.n, 1:] = g
        parts = [torch.empty_like(buf) for _ in range(self.world)]
        dist.all_gather(parts, buf, group=self.group)
        rows = torch.cat([p[:n] for p, (_, n) in zip(parts, self.rows)], dim=0).to(self.engine_device)
        return rows[:, 0].contiguous(), rows[:, 1:].contiguous()

    def step(self):
        """One SMC^2 iteration; returns the engine's statistics (identical on every rank)."""
        if self.stream is not None:
            with torch.cuda.stream(self.stream):
                ll, g = self.engine.step_filters(self.row0, self.n)
                ll_all, g_all = self._exchange(ll, g)
        else:
            ll, g = self.engine.step_filters(self.row0, self.n)
            ll_all, g_all = self._exchange(ll, g)
        return self.engine.step_update(ll_all, g_all)
