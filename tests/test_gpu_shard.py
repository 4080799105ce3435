"""The sharded design on the GPU engine: the network split into shard models
(own cells, every connection into them, stubs for remote presynaptic cells)
that advance one min-delay epoch each and exchange the epoch's spikes through
the host (pa_read_spikes, then pa_inject_spikes into the other shards).  The
shards run one after another in one process on one GPU -- no kernel waits on
another -- and must equal the single model bit for bit in FP64."""
import numpy as np
import pytest

from paper_2411_16445_b300 import engine as E
from paper_2411_16445_b300 import shard as S
from paper_2411_16445_b300 import workloads as W

from _nets import tiny_tree_net

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_ranks", [2, 3])
@pytest.mark.parametrize("which", ["stc", "trees"])
def test_shards_equal_the_whole_network(which, n_ranks):
    if which == "stc":
        net = W.recurrent_stc(n_exc=80, n_inh=20, p=0.1, w_bg=3e-3, bg_rate=20.0)
    else:
        net = tiny_tree_net(n_cells=90)
    Es = S.epoch_steps(net)
    n_epochs = 60
    whole = E.Model(net, precision=E.PA_FP64)
    whole.advance(n_epochs * Es * net.dt)
    whole.sync()
    shards, runs = S.run_local_shards(
        net, n_ranks, lambda sh, Ee: E.Model(sh.net, precision=E.PA_FP64, max_epoch_steps=Ee),
        n_epochs)
    ncv = net.cell_ncv()
    off = np.r_[0, np.cumsum(ncv)]
    v_all = whole.read_state(E.FIELD_V)
    g, s, t = whole.read_spikes()
    w_all = whole.read_weights()
    n_spk = 0
    for sh, run in zip(shards, runs):
        run.sim.sync()
        v_ref = np.concatenate([v_all[off[c]:off[c + 1]] for c in sh.own])
        assert np.array_equal(v_ref, run.sim.read_state(E.FIELD_V)[:len(v_ref)])
        sel = np.isin(g, sh.own)
        gg, ss, tt = run.own_spikes()
        assert np.array_equal(g[sel], gg) and np.array_equal(s[sel], ss)
        assert np.array_equal(t[sel], tt)
        assert np.array_equal(w_all[sh.conn], run.sim.read_weights())
        n_spk += len(gg)
    assert n_spk == len(g) > 50


def test_inject_spikes_rejects_steps_outside_the_last_epoch():
    net = W.recurrent_stc(n_exc=80, n_inh=20, p=0.1, w_bg=3e-3, bg_rate=20.0)
    m = E.Model(net, precision=E.PA_FP64)
    Es = m.info().epoch_steps
    m.advance(3 * Es * net.dt)
    with pytest.raises(E.PaError) as ei:
        m.inject_spikes(np.array([1], np.int32), np.array([3 * Es], np.int64))  # not past
    assert ei.value.code == -1
    with pytest.raises(E.PaError):
        m.inject_spikes(np.array([1], np.int32), np.array([Es], np.int64))      # too old
    with pytest.raises(E.PaError):
        m.inject_spikes(np.array([net.n_cells], np.int32), np.array([2 * Es], np.int64))
    m.inject_spikes(np.array([1, 2], np.int32), np.array([2 * Es, 3 * Es - 1], np.int64))
    m.advance(4 * Es * net.dt)
    m.sync()
