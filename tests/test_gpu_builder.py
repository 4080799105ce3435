"""The host model builder through the C-ABI: its parallel phases (CV
discretisation, synapse ordering, run flags, connection validation) give the
same model with one host thread as with every core, and of several bad
connections the lowest-indexed one is reported."""
import numpy as np
import pytest

from paper_2411_16445_b300 import engine as E
from paper_2411_16445_b300 import workloads as W

from _nets import tiny_tree_net

pytestmark = pytest.mark.gpu


def _state(net, precision, flags, steps):
    m = E.Model(net, precision=precision, flags=flags)
    info = m.info()
    m.advance(steps * net.dt)
    out = (m.read_state(E.FIELD_V), m.read_spikes()[1], m.read_weights())
    m.close()
    return (info.n_cv, info.n_padded_cv, info.n_static_cv, info.n_wide), out


@pytest.mark.parametrize("precision", [E.PA_FP64, E.PA_MIXED])
@pytest.mark.parametrize("which", ["trees", "busyring_stdp", "recurrent_stc_noise"])
def test_build_threads_do_not_change_the_model(precision, which):
    net = {"trees": lambda: tiny_tree_net(n_cells=300),
           "busyring_stdp": lambda: W.busyring(n_cells=64, depth=2, s=100, stdp=True),
           "recurrent_stc_noise": lambda: W.recurrent_stc(n_exc=96, n_inh=24,
                                                          sigma_pl=2.90436)}[which]()
    a_info, a = _state(net, precision, E.FLAG_BUILD_THREADS(1), 600)
    for flags in (0, E.FLAG_BUILD_THREADS(3)):
        b_info, b = _state(net, precision, flags, 600)
        assert a_info == b_info
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_lowest_bad_connection_is_reported():
    net = W.recurrent_stc(n_exc=160, n_inh=40)
    n = net.n_conn
    cases = [
        ("conn_cv", [n - 3, n // 3], [50, 50], f"connection {n // 3}: bad dst_cv"),
        ("conn_dst", [n // 2, 17], [-1, net.n_cells], "connection 17: bad dst_gid"),
        ("conn_delay", [n - 1, n // 5], [0.0, 0.0],
         f"connection {n // 5}: delay must be at least one step"),
    ]
    for field, idx, val, msg in cases:
        bad = W.recurrent_stc(n_exc=160, n_inh=40)
        arr = getattr(bad, field).copy()
        arr[idx] = val
        setattr(bad, field, arr)
        with pytest.raises(E.PaError) as ei:
            E.Model(bad)
        assert ei.value.code == -1
        assert msg in str(ei.value)
