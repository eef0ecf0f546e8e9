"""Host logic of the multi-GPU path, on CPU with the gloo backend (world
size 2): ranks split an ensemble of independent networks without overlap,
and the whole-job rate is (segments of all ranks) / (slowest rank's time)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = bench.rank_configs(64, world, rank)
    segs = 1000.0 * (rank + 1) * len(mine)   # different work per rank
    ms = 10.0 * (rank + 1)                    # rank 1 is the slower one
    rate, tot_segs, tot_ms = bench.global_rate(segs, ms)
    q.put((rank, mine, rate, tot_segs, tot_ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_and_rate():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, rate0, s0, t0), (r1, m1, rate1, s1, t1) = out
    assert sorted(m0 + m1) == list(range(64)) and not set(m0) & set(m1)
    assert s0 == s1 == 1000.0 * len(m0) + 2000.0 * len(m1)
    assert t0 == t1 == 20.0
    assert abs(rate0 - s0 / 0.02) < 1e-6 and rate0 == rate1
