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


def _worker_forces(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist

    import bench
    import oracle
    from paper_1712_07739_gb300 import synth

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nets = synth.ensemble(n_configs=6, ns_range=(60, 150), seed=9)  # every rank draws the same ensemble
    mat = oracle.Material.iso(1.0, 0.3)
    mine = bench.rank_configs(len(nets), world, rank)
    local = {k: oracle.network_forces(mat, *nets[k], nthreads=1)[0] for k in mine}
    segs = float(sum(len(nets[k][1]) for k in mine))
    rate, tot_segs, tot_ms = bench.global_rate(segs, 5.0 + rank)
    parts = [None] * world
    dist.all_gather_object(parts, local)
    if rank == 0:
        merged = {}
        for p in parts:
            assert not set(p) & set(merged)  # no network computed twice
            merged.update(p)
        q.put((sorted(merged), {k: v.tolist() for k, v in merged.items()}, tot_segs, tot_ms, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_compute_their_shard_of_an_ensemble():
    """Each rank evaluates the nodal forces of its share of a 6-network
    ensemble (the oracle stands in for the GPU pass on CPU); the gathered
    forces equal a single-process evaluation of every network, and the job
    rate counts every network's segments over the slowest rank's time."""
    import multiprocessing as mp

    import numpy as np

    import oracle
    from paper_1712_07739_gb300 import synth

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_forces, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    keys, forces, tot_segs, tot_ms, rate = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    nets = synth.ensemble(n_configs=6, ns_range=(60, 150), seed=9)
    assert keys == list(range(6))
    mat = oracle.Material.iso(1.0, 0.3)
    for k, (n, s, b) in enumerate(nets):
        F, _ = oracle.network_forces(mat, n, s, b, nthreads=1)
        assert np.array_equal(np.array(forces[k]), F)
    assert tot_segs == sum(len(s) for _, s, _ in nets)
    assert tot_ms == 6.0 and abs(rate - tot_segs / 0.006) < 1e-6
