"""Batches: resident models advanced together, one grouped time-step launch
per epoch over all of them.  Every member's results must equal the same model
advanced alone, bit for bit, in every precision and for chains and trees --
with members joining late, leaving early and being advanced alone in
between."""
import numpy as np
import pytest

from paper_2411_16445_b300 import engine as E
from paper_2411_16445_b300 import workloads as W

from _nets import tiny_tree_net

pytestmark = pytest.mark.gpu


def jobs(kind):
    if kind == "chains":
        return [W.serving_job(n, long_d, L, d, seed, dt=0.2)
                for n, long_d, L, d, seed in ((1, True, 300.0, 1.0, 1), (37, False, 150.0, 0.7, 2),
                                              (300, True, 640.0, 1.8, 3), (1200, False, 420.0, 1.2, 4),
                                              (65, True, 100.0, 0.5, 5))]
    return [tiny_tree_net(n_cells=n, seed=s) for n, s in ((45, 5), (70, 6), (33, 7))]


def state(m):
    m.sync()
    return (m.read_state(E.FIELD_V), m.read_spikes(), m.read_weights())


def same(a, b):
    assert np.array_equal(a[0], b[0])
    for x, y in zip(a[1], b[1]):
        assert np.array_equal(x, y)
    assert np.array_equal(a[2], b[2])


@pytest.mark.parametrize("precision", [E.PA_FP64, E.PA_MIXED, E.PA_FP32])
@pytest.mark.parametrize("kind", ["chains", "trees"])
def test_batch_members_equal_models_alone(kind, precision):
    nets = jobs(kind)
    flags = E.FLAG_NARROW_ONLY
    alone = []
    for j, net in enumerate(nets):
        m = E.Model(net, precision=precision, flags=flags)
        Es = m.info().epoch_steps
        m.advance((40 + 8 * j) * Es * net.dt)
        alone.append(state(m))
        m.close()
    b = E.Batch()
    ms = [E.Model(net, precision=precision, flags=flags) for net in nets]
    Es = [m.info().epoch_steps for m in ms]      # a 1-cell job has no recurrent delay: 64
    # member 0 starts alone, the others join; members leave as they finish
    ms[0].advance(5 * Es[0] * nets[0].dt)
    for m in ms[:-1]:
        b.add(m)
    b.advance_epochs(11)             # 8-epoch graph + 1-epoch graphs
    b.add(ms[-1])                    # joins late (at step 0)
    b.advance_epochs(9)
    b.remove(ms[1])                  # leaves, runs alone for a while, rejoins
    ms[1].advance((ms[1].step + 3 * Es[1]) * nets[1].dt)
    b.add(ms[1])
    done = set()
    while len(done) < len(ms):
        b.advance_epochs(1)
        for j, m in enumerate(ms):
            if j in done:
                continue
            target = (40 + 8 * j) * Es[j]
            if m.step >= target:
                assert m.step == target
                b.remove(m)
                same(alone[j], state(m))
                done.add(j)
    assert b.info()["graph_launches"] > 0


def test_batch_rejects_mismatched_members():
    a = E.Model(jobs("chains")[1], precision=E.PA_MIXED, flags=E.FLAG_NARROW_ONLY)
    b = E.Model(jobs("chains")[2], precision=E.PA_FP64, flags=E.FLAG_NARROW_ONLY)
    t = E.Model(jobs("trees")[0], precision=E.PA_MIXED, flags=E.FLAG_NARROW_ONLY)
    bt = E.Batch()
    bt.add(a)
    for m in (b, t):
        with pytest.raises(E.PaError):
            bt.add(m)
    with pytest.raises(E.PaError):
        bt.add(a)
    a.advance(3 * a.dt)              # off its epoch boundary
    with pytest.raises(E.PaError):
        bt.advance_epochs(1)
