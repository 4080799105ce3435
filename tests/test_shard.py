"""The sharded design (one network over several GPUs, one rank per GPU) on the
host: each rank holds its cells, every connection into them and passive stubs
for remote presynaptic cells, advances one min-delay epoch, and the ranks
all-gather the epoch's spikes {gid, step}, each injecting the remote ones into
its model.  Checked with the FP64 oracle as each rank's model: two gloo ranks
(a real all-gather across processes), and three ranks in one process, against
the single-model oracle bit for bit (voltages, spikes with their times, plastic
weights and tags).  Not measured on hardware: every run here has one GPU."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

import oracle as O
from paper_2411_16445_b300 import shard as S
from paper_2411_16445_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_EPOCHS = 40


def small_net():
    return W.recurrent_stc(n_exc=40, n_inh=10, p=0.2, w_bg=3e-3, bg_rate=20.0)


class OracleSim:
    """The oracle behind the interface ShardedRun drives."""

    def __init__(self, net):
        self.o = O.Oracle(net)
        self.n_read = 0

    def advance_steps(self, n):
        self.o.run(n)

    def read_spikes(self):
        g, s, t = self.o.spikes()
        out = (g[self.n_read:].astype(np.int64), s[self.n_read:], t[self.n_read:])
        self.n_read = len(g)
        return out

    def inject_spikes(self, g, s):
        self.o.inject_spikes(g, s)


def reference(net, steps):
    o = O.Oracle(net)
    o.run(steps)
    return o


def check_rank(net, ref, sh, sim, run):
    """The rank's own cells and connections against the single-model oracle."""
    ncv = net.cell_ncv()
    off = np.r_[0, np.cumsum(ncv)]
    v_ref = np.concatenate([ref.v()[off[c]:off[c + 1]] for c in sh.own])
    v_sh = sim.o.v()[:int(ncv[sh.own].sum())]
    assert np.array_equal(v_ref, v_sh)
    g, s, t = ref.spikes()
    sel = np.isin(g, sh.own)
    o = np.lexsort((g[sel], s[sel]))
    gg, ss, tt = run.own_spikes()
    assert np.array_equal(g[sel][o], gg) and np.array_equal(s[sel][o], ss)
    assert np.array_equal(t[sel][o], tt)
    for f in (O.SYN_WEIGHT_TOTAL, O.SYN_H, O.SYN_Z, O.SYN_C, O.SYN_G):
        assert np.array_equal(ref.syn(f)[sh.conn], sim.o.syn(f))
    return len(gg)


def test_partition_and_shard_networks():
    net = small_net()
    parts = S.partition(net, 3)
    assert np.array_equal(np.concatenate(parts), np.arange(net.n_cells))
    E = S.epoch_steps(net)
    assert E == 15                                      # 3 ms at dt 0.2 ms
    seen = []
    for own in parts:
        sh = S.shard_network(net, own)
        seen.append(sh.conn)
        assert np.all(np.isin(net.conn_dst[sh.conn], own))
        assert np.all(np.diff(sh.conn) > 0)            # the whole network's order
        assert sh.net.n_cells == len(own) + len(sh.stubs)
        assert not np.any(np.isin(sh.stubs, own))
        # every remote presynaptic cell has its stub, and sources map back
        src = net.conn_src[sh.conn]
        loc = sh.net.conn_src
        assert np.array_equal(loc >= 0, src >= 0)
        back = np.r_[sh.own, sh.stubs]
        assert np.array_equal(back[loc[loc >= 0]], src[src >= 0])
    assert np.array_equal(np.sort(np.concatenate(seen)), np.arange(net.n_conn))


def test_three_shards_in_one_process_equal_the_whole_network():
    net = small_net()
    E = S.epoch_steps(net)
    ref = reference(net, N_EPOCHS * E)
    assert len(ref.spikes()[0]) > 50
    shards, runs = S.run_local_shards(net, 3, lambda sh, E: OracleSim(sh.net), N_EPOCHS)
    n = sum(check_rank(net, ref, sh, run.sim, run) for sh, run in zip(shards, runs))
    assert n == len(ref.spikes()[0])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), OMP_NUM_THREADS="1")
    import torch.distributed as dist
    from test_shard import OracleSim, check_rank, reference, small_net
    from paper_2411_16445_b300 import shard as S
    dist.init_process_group("gloo", rank=rank, world_size=ws)

    def allgather(obj):
        lst = [None] * ws
        dist.all_gather_object(lst, obj)
        return lst

    net = small_net()
    E = S.epoch_steps(net)
    sh = S.shard_network(net, S.partition(net, ws)[rank])
    sim = OracleSim(sh.net)
    run = S.ShardedRun(sh, sim, E, allgather)
    run.advance_epochs(N_EPOCHS)
    ref = reference(net, N_EPOCHS * E)
    try:
        out[rank] = ("ok", check_rank(net, ref, sh, sim, run), len(sh.stubs))
    except AssertionError as e:
        out[rank] = ("fail", str(e), 0)
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_the_whole_network():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True,
                       start_method="spawn")
    ref = reference(small_net(), N_EPOCHS * 15)
    assert out[0][0] == "ok" and out[1][0] == "ok", (out[0], out[1])
    assert out[0][1] + out[1][1] == len(ref.spikes()[0])
    assert out[0][2] > 0 and out[1][2] > 0            # spikes did cross the ranks
