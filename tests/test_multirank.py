"""The multi-GPU host logic of bench.py on two CPU ranks (gloo, 127.0.0.1):
the job time is the slowest rank's, every rank correlates its own arrays,
and the job's units are the sum over ranks.  No GPU is involved."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from synth import voltgen as vg


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + rank * 5.0, world, device="cpu")
        idx = bench.rank_array_index(1, rank)
        head = vg.gauss3(vg.gauss3_params(1503, 16, 4, array=idx), 0, 8)
        out[rank] = (t, idx, head.tobytes())
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_own_data():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] != res[1][1]
    assert res[0][2] != res[1][2]          # different data on each rank
    assert bench.job_units(1000, 3, world) == 6000


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.5, 1) == 3.5
