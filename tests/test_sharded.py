"""Row partition and exchange of the sharded SMC^2 sampler, on CPU gloo ranks.

The sampler is run by two processes, each filtering half of the N samples; the result must
equal, exactly, the one-process oracle run (the oracle's arithmetic per row does not depend
on which process computes it, and the outer update sees the same N rows)."""
import multiprocessing as mp
import socket

import numpy as np
import pytest

from paper_2407_17296_gb300.sharded import shard_rows


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("N", [0, 1, 2, 7, 64, 1023])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_rows_partition(N, world):
    blocks = [shard_rows(N, world, r) for r in range(world)]
    nxt = 0
    for row0, n in blocks:
        assert row0 == nxt and n >= 0
        nxt = row0 + n
    assert nxt == N
    sizes = [n for _, n in blocks]
    assert max(sizes) - min(sizes) <= 1


def test_shard_rows_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard_rows(10, 2, 2)


@pytest.mark.parametrize("N", [8, 7])
def test_two_gloo_ranks_equal_one_process(N):
    from oracle import smc2 as osmc2
    from paper_2407_17296_gb300 import workloads
    from .sharded_oracle_engine import worker

    K = 3
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, N, K, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(2)], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(r[1], r[2]) for r in res] == [shard_rows(N, 2, 0), shard_rows(N, 2, 1)]

    w = workloads.lg1(T=12, N=N, M=32, K=K)
    records, _ = osmc2.run(w.family, w.dx, w.dy, w.H, w.y, N, w.M, K, w.gamma, w.proposal, w.seed,
                           D=w.D)
    last = records[-1]
    theta = last["theta"][last["ancestors"]] if last["resampled"] else last["theta"]
    for r in res:
        np.testing.assert_array_equal(r[3], theta)
        assert [s[0] for s in r[6]] == [rec["k"] for rec in records]
        assert [s[1] for s in r[6]] == [rec["ess"] for rec in records]
        assert [s[2] for s in r[6]] == [rec["resampled"] for rec in records]
    np.testing.assert_array_equal(res[0][4], res[1][4])
    np.testing.assert_array_equal(res[0][5], res[1][5])
