"""The multi-GPU path of bench.py is replicas only: each rank simulates the same
network structure with its own drive seed (independent Poisson input), ranks
exchange nothing on the data path, and the job's time is the slowest rank's.
Checked here with two gloo ranks on CPU."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    w, r, _ = bench.dist_setup()
    net = bench.workload(64, 16, seed_offset=r)
    ms, value = bench.replica_total(10.0 * (r + 1), 1000.0, w)
    out[rank] = (w, r, int(net.seed), int(net.conn_src.sum()), ms, value)
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True,
                       start_method="spawn")
    a, b = out[0], out[1]
    assert a[:2] == (2, 0) and b[:2] == (2, 1)
    assert a[2] != b[2] and a[3] == b[3]          # same structure, own drive seed
    # the job time is the slowest rank's; the value counts both ranks' work
    for r in (a, b):
        assert r[4] == 20.0 and np.isclose(r[5], 2 * 1000.0 / 20e-3)
