"""Multi-GPU form of the bench (replicas): disjoint property streams per rank
and the max-time / summed-nodes reduction, run as world-size-2 gloo ranks on
the CPU (the data path has no collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    layers = synth.make_network(1)
    # each rank draws its own properties: disjoint seeds, hence different images
    pr = synth.make_properties(1, layers, n=2, start=bench.rank_start(rank))
    ms, nodes = bench.reduce_timing(10.0 + rank, 100 * (rank + 1))
    q.put((rank, [float(p.x0.sum()) for p in pr], ms, nodes))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_reduce_and_shard():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, x0, ms0, n0), (r1, x1, ms1, n1) = out
    assert ms0 == ms1 == 11.0            # max over ranks
    assert n0 == n1 == 300               # nodes summed over ranks
    assert set(x0).isdisjoint(x1)        # disjoint property streams


def test_single_process_is_identity():
    import bench
    assert bench.reduce_timing(3.5, 7) == (3.5, 7)
    assert bench.rank_start(0) == 0 and bench.rank_start(3) == 3 * bench.RANK_STRIDE
