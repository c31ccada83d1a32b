"""The multi-GPU path of the benchmark is replicas only: each rank advances
its own copy of the workload (its own seeded mesh) and the ranks meet once,
in the max-over-ranks reduction of the timed region.  This runs that host
logic as two gloo ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_2106_06280_gb300 import workloads as W

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, rk, _ = bench.dist_info()
    ms = 10.0 + 5.0 * rk  # rank 1 is the slower one
    ms_max = bench.max_over_ranks(ms, "cpu")
    mesh = W.double_mach(24, 6, seed=bench.replica_seed(rk)).mesh
    out[rank] = (ws, rk, ms_max, bench.whole_job_rate(1000.0, ws, ms_max), float(mesh.xy.sum()), mesh.nc)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_max_time_and_whole_job_rate():
    import torch.multiprocessing as mp

    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork after the oracle's threads exist
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        r0, r1 = out[0], out[1]
    assert r0[0] == r1[0] == 2 and (r0[1], r1[1]) == (0, 1)
    assert r0[2] == r1[2] == 15.0  # both ranks see the slowest rank's time
    assert r0[3] == pytest.approx(2 * 1000.0 / 15e-3)  # all ranks' units over the slowest time
    assert r0[5] == r1[5] and r0[4] != r1[4]  # same workload size, independent seeded meshes
