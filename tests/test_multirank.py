"""The N > 1 path of bench.py on CPU: two gloo ranks (no GPU).

Independent problems shard across ranks with no collective on the data path; the only collectives
are the barrier and the max-over-ranks reduction of the step time. Checked here: every rank gets the
maximum, a single process needs no process group, and the ranks' problems (random splits, batches)
are distinct and reproducible.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        dist.barrier()
        got = bench.max_over_ranks(10.0 * (rank + 1), torch.device("cpu"))
        p = bench.rank_problem("d256_k8", rank)
        out[rank] = (got, float(np.asarray(p.X).sum()), bench.rank_batch_seed(rank))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_sharding_with_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 20.0
    assert out[0][1] != out[1][1]                 # each rank solves its own split
    assert out[0][2] != out[1][2]                 # and its own batch


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    a = bench.rank_problem("d256_k8", 0)
    b = bench.rank_problem("d256_k8", 0)
    assert np.array_equal(a.X, b.X)
