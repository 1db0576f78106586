"""The multi-GPU bookkeeping (replicas, max time over ranks, summed work) on
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2603_11189_gb300 import replicas
    w, r, lr = replicas.world()
    # rank r processed 1000*(r+1) units in 10*(r+1) ms
    value, ms = replicas.throughput(1000.0 * (r + 1), 10.0 * (r + 1))
    out[r] = (w, r, value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_throughput_uses_slowest_rank_and_all_units():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        w, rr, value, ms = out[r]
        assert w == world and rr == r
        assert ms == pytest.approx(20.0)                 # max over ranks
        assert value == pytest.approx(3000.0 / 0.020)   # all units / slowest time
