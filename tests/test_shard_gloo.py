"""Sample sharding across ranks (host logic), world size 2 over gloo on CPU.

Each rank takes its Philox index window from shard_range, classifies it (the
oracle stands in for the GPU here), and the int64 counts are summed with
combine_counts; the result must equal one process over the whole range.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_per_rank, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads as W
    from oracle import oracle as O
    from paper_2604_17066_gb300.shard import combine_counts, shard_range
    p = W.c1_grid()
    off, n = shard_range(n_per_rank, rank, world, offset=1000)
    X = O.sample(p.pmf, 1, off, n)
    lab, cnt = O.classify(X, p.ref_L, p.ref_U)
    C = O.grad_counts(X, lab, p.K)
    t = torch.from_numpy(np.concatenate([cnt, C.ravel()]).astype(np.int64))
    combine_counts(t)
    if rank == 0:
        out.put(t.numpy().tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_counts_equal_one_process():
    world, n_per_rank = 2, 6000
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_per_rank, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    combined = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    import workloads as W
    from oracle import oracle as O
    p = W.c1_grid()
    X = O.sample(p.pmf, 1, 1000, world * n_per_rank)
    lab, cnt = O.classify(X, p.ref_L, p.ref_U)
    C = O.grad_counts(X, lab, p.K)
    assert combined == np.concatenate([cnt, C.ravel()]).tolist()


def test_shard_range_partitions_the_stream():
    from paper_2604_17066_gb300.shard import shard_range
    spans = [shard_range(100, r, 4, offset=7) for r in range(4)]
    assert spans == [(7, 100), (107, 100), (207, 100), (307, 100)]
    with pytest.raises(ValueError):
        shard_range(100, 4, 4)
