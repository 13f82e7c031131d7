"""Host logic of multi-rank runs, tested with gloo on CPU (world size 2):
LP sharding (no data-path collective) and the max-over-ranks timing."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    ms = [12.5, 40.0][rank]
    units = [100, 156][rank]
    q.put((rank, bench.reduce_over_ranks(ms, units, torch.device("cpu"))))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0] == out[1] == (40.0, 256.0)


def test_shard_lps_partitions_and_balances():
    sys.path.insert(0, ROOT)
    import bench
    w = [5, 1, 9, 3, 3, 7, 2, 8]
    for ws in (1, 2, 3):
        parts = bench.shard_lps(w, ws)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(w)))
        loads = [sum(w[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(w)
    assert bench.shard_lps(w, 2) == bench.shard_lps(w, 2)  # deterministic
