"""Multi-rank host logic on CPU: two gloo ranks shard a node batch, bound their
shards with the oracle, and gather; the result equals the single-process one.
(The CUDA path shards the same way; one GPU per rank, no data-path collective.)"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2507_20769_gb300 import shard


def test_shard_range_partitions_exactly():
    for n in (0, 1, 5, 64, 1001):
        for w in (1, 2, 3, 8):
            spans = [shard.shard_range(n, r, w) for r in range(w)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(w - 1))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2507_20769_gb300 import workloads as W
        t = W.config_tape(1)
        boxes = W.bisection_frontier(t.root_box, 7, seed=4)
        b, e = shard.shard_range(len(boxes), rank, world)
        r = oracle.bound_nodes(t, boxes[b:e], [4, 4], grad_mode="forward")
        lb = shard.gather_node_results(r["lb"], len(boxes))
        hull = shard.gather_node_results(np.stack([r["minlo"][:, 0], r["maxhi"][:, 0]], 1), len(boxes))
        tmax = shard.max_over_ranks(float(rank + 1))
        tsum = shard.sum_over_ranks(float(e - b))
        q.put((rank, lb, hull, tmax, tsum))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_gather():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    from paper_2507_20769_gb300 import workloads as W
    t = W.config_tape(1)
    boxes = W.bisection_frontier(t.root_box, 7, seed=4)
    ref = oracle.bound_nodes(t, boxes, [4, 4], grad_mode="forward")
    for rank, lb, hull, tmax, tsum in res:
        assert np.array_equal(lb, ref["lb"])
        assert np.array_equal(hull[:, 0], ref["minlo"][:, 0]) and np.array_equal(hull[:, 1], ref["maxhi"][:, 0])
        assert tmax == 2.0 and tsum == 7.0
