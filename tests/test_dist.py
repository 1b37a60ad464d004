"""The N > 1 path on CPU: two gloo ranks shard 64 uneven slices (disjoint, complete,
balanced) and reduce timings with max/sum; no data crosses ranks on the solve path."""
import os
import socket

import pytest

from paper_1810_03275_gb300 import dist


def _costs():
    import numpy as np
    rng = np.random.default_rng(11)
    sizes = (256, 384, 512, 768, 1024)
    return [float(sizes[rng.integers(0, 5)] ** 2 * rng.integers(180, 1441)) for _ in range(64)]


def test_shard_partitions_and_balances():
    costs = _costs()
    for ws in (1, 2, 3, 4, 8):
        parts = [dist.shard(costs, r, ws) for r in range(ws)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= 1.1 * (sum(costs) / ws) + max(costs)


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist_
    r, w, _ = dist.init(backend="gloo")
    mine = dist.shard(_costs(), r, w)
    t_max = dist.max_over_ranks(1.0 + r)
    n_all = dist.sum_over_ranks(len(mine))
    dist.barrier()
    q.put((r, mine, t_max, n_all))
    dist_.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, n0), (r1, m1, t1, n1) = res
    assert set(m0).isdisjoint(m1) and sorted(m0 + m1) == list(range(64))
    assert t0 == t1 == 2.0 and n0 == n1 == 64
