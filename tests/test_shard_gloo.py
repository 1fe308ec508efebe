"""Multi-rank host logic on CPU: two gloo ranks shard a node batch, process
their shards, and gather; the result equals the single-process one. One test
bounds the shards with the oracle; the other drives the library's own host
path on each shard (split picking, constraint propagation and the gradient
enclosure behind the B&B's descent corner -- the work a rank's host does
around its GPU launches) and checks the gathered results against the oracle.
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


def _host_path_shard(rank, world, t, boxes):
    """the library's host path on this rank's shard of the node batch"""
    from paper_2507_20769_gb300 import ivb
    b, e = shard.shard_range(len(boxes), rank, world)
    ref_w = t.root_box[:, 1] - t.root_box[:, 0]
    splits = np.stack([ivb.ivb_pick_splits(bx, 1 << 12, "adaptive", ref_w) for bx in boxes[b:e]]).astype(np.float64)
    tight, inf = ivb.ivb_propagate(t, boxes[b:e], ub=float("inf"), passes=3)
    grads = np.stack([np.stack([ivb.ivb_host_gradient(t, bx, o, "adjoint") for o in range(t.n_out)])
                      for bx in boxes[b:e]])
    return splits, tight, inf.astype(np.float64), grads


def _host_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2507_20769_gb300 import build as B
        B.build()
        import problems as P
        t = P.rational_tape_for_shards()
        boxes = P.shard_boxes(t)
        splits, tight, inf, grads = _host_path_shard(rank, world, t, boxes)
        n = len(boxes)
        q.put((rank, shard.gather_node_results(splits, n), shard.gather_node_results(tight, n),
               shard.gather_node_results(inf, n), shard.gather_node_results(grads, n)))
    except Exception as e:          # report instead of leaving the parent waiting
        q.put((rank, repr(e)))
        raise
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_drive_the_library_host_path():
    """each rank runs ivb_pick_splits, ivb_propagate and ivb_host_gradient on
    its shard; gathered, they equal one process's results and, on this
    rational tape, the oracle's bit for bit"""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_host_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    assert all(len(r) == 5 for r in res), [r for r in res if len(r) != 5]
    assert all(p.exitcode == 0 for p in procs)
    import oracle
    import problems as P
    t = P.rational_tape_for_shards()
    boxes = P.shard_boxes(t)
    one = _host_path_shard(0, 1, t, boxes)
    ref_w = t.root_box[:, 1] - t.root_box[:, 0]
    o_splits = np.stack([oracle.pick_splits(bx, 1 << 12, "adaptive", ref_w) for bx in boxes])
    o_tight, o_inf = oracle.propagate(t, boxes, passes=3)
    o_grads = np.stack([oracle.gradient(t, bx, "adjoint") for bx in boxes])
    for rank, splits, tight, inf, grads in res:
        for got, single in zip((splits, tight, inf, grads), one):
            assert np.array_equal(got, single)
        assert np.array_equal(splits, o_splits.astype(np.float64))
        assert np.array_equal(tight, o_tight) and np.array_equal(inf.astype(bool), o_inf.astype(bool))
        assert np.array_equal(grads, o_grads)
