"""Multi-rank host logic on CPU (gloo, world size 2): shard assignment covers
the transmitters exactly once, and the timing reductions bench.py uses give
the max / sum over ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2303_11103_gb300.shard import max_over_ranks, shard_range, sum_over_ranks


def test_shard_range_partitions():
    for n in (0, 1, 7, 64, 1000):
        for w in (1, 2, 3, 8):
            got = [shard_range(n, r, w) for r in range(w)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(got[i][1] == got[i + 1][0] for i in range(w - 1))
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(5, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, e = shard_range(64, rank, world)
    mx = max_over_ranks(10.0 * (rank + 1))
    sm = sum_over_ranks(e - b)
    dist.barrier()
    q.put((rank, b, e, mx, sm))
    dist.destroy_process_group()


def test_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(b, e) for _, b, e, _, _ in res] == [(0, 32), (32, 64)]
    assert all(mx == 20.0 and sm == 64 for _, _, _, mx, sm in res)
