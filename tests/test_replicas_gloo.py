"""Multi-rank host logic of the energy-replica runs, exercised with two gloo ranks on CPU:
energy ownership is a partition, ranks pick different batches, and the timed region's
max-over-ranks reduction returns the slowest rank's time."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    import torch.distributed as dist

    from paper_2508_19138_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b, e = replicas.energy_slice(rank, world, 513)
        t = 1.5 + rank  # rank 1 is "slower"
        dist.barrier()
        tmax = replicas.max_over_ranks(t, dist)
        total = replicas.sum_over_ranks(e - b, dist)
        results[rank] = (b, e, tmax, total, replicas.batch_index(rank, 3, 32))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.spawn(_worker, args=(world, port, results), nprocs=world, join=True)
        res = dict(results)
    (b0, e0, t0, n0, k0), (b1, e1, t1, n1, k1) = res[0], res[1]
    assert (b0, e0) == (0, 257) and (b1, e1) == (257, 513)
    assert t0 == t1 == 2.5
    assert n0 == n1 == 513
    assert k0 != k1


def test_energy_slice_partition_single_process():
    from paper_2508_19138_gb300 import replicas
    for world in (1, 2, 3, 8):
        seen = []
        for r in range(world):
            b, e = replicas.energy_slice(r, world, 100)
            seen.extend(range(b, e))
        assert seen == list(range(100))
    with pytest.raises(ValueError):
        replicas.energy_slice(2, 2, 10)
    assert replicas.max_over_ranks(3.0) == 3.0
