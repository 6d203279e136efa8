"""Replicas: world-size-2 gloo processes on CPU run independent oracle chains and aggregate
time (max) and work (sum) the way the benchmark does on GPUs."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, outdir):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_1208_0166_gb300.replicas import aggregate, replica_seed

    seed = replica_seed(5, rank)
    lat = O.Lattice(4, 4, 1.0, seed)
    lat.sweep(1, 1)
    secs = 1.0 + rank          # stand-in local times
    units = 100.0 * (rank + 1)  # stand-in local work
    dist.barrier()
    t, u = aggregate(secs, units, dist)
    np.save(os.path.join(outdir, f"r{rank}.npy"), np.concatenate([[seed, t, u], lat.theta[:8]]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_aggregate_max_time_and_total_work(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0, r1 = np.load(tmp_path / "r0.npy"), np.load(tmp_path / "r1.npy")
    assert r0[0] == 5 and r1[0] == 6                  # distinct chains
    assert r0[1] == r1[1] == 2.0                      # slowest rank's time
    assert r0[2] == r1[2] == 300.0                    # work summed over ranks
    assert not np.array_equal(r0[3:], r1[3:])         # independent configurations


def test_single_process_aggregate_is_identity():
    from paper_1208_0166_gb300.replicas import aggregate, replica_seed

    assert aggregate(1.5, 7.0) == (1.5, 7.0)
    assert replica_seed(1, 0) == 1 and replica_seed(1, 3) == 4
