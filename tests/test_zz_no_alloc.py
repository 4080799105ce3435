"""pa_advance_noalloc: advancing a model without any GPU allocation during the call.

It is meant for callers that must not allocate device memory while they run --
code whose allocations belong to another memory manager, or a real-time host
thread where an allocation could stall or fail.  Its epoch kernels take the
Hines elimination scratch from one fixed device array of the library instead
of from the model.  These tests check, through the C-ABI, that calls in a row
give the same results as pa_advance, bit for bit in every precision (the same
kernels run; only the scratch pointers differ), including after other models
have left the shared array dirty; that device memory is unchanged across the
calls; and that too-large models and replay mode are refused with an error.
The file is named so that pytest collects it last; it also passes when run
alone in a fresh process."""
import numpy as np
import pytest

from paper_2411_16445_b300 import engine as E
from paper_2411_16445_b300 import workloads as W

from _nets import hca_tree_net, tiny_tree_net

pytestmark = pytest.mark.gpu


def small_net():
    return W.recurrent_stc(n_exc=80, n_inh=20, p=0.1, w_bg=3e-3, bg_rate=20.0)


def assert_same(ref, new):
    ref.sync()
    new.sync()
    assert np.array_equal(ref.read_state(E.FIELD_V), new.read_state(E.FIELD_V))
    for a, b in zip(ref.read_spikes(), new.read_spikes()):
        assert np.array_equal(a, b)
    assert np.array_equal(ref.read_weights(), new.read_weights())


@pytest.mark.parametrize("precision", [E.PA_FP64, E.PA_MIXED, E.PA_FP32])
def test_noalloc_matches_advance_on_two_calls(precision):
    net = small_net()
    ref = E.Model(net, precision=precision)
    new = E.Model(net, precision=precision)
    for t_end in (40 * net.dt * 7 + 3 * net.dt, 40 * net.dt * 19):  # partial, then whole epochs
        ref.advance(t_end)
        new.advance_noalloc(t_end)
        assert_same(ref, new)


def test_noalloc_after_other_models_dirtied_the_array():
    """Models with wide cells, a diffusing PRP field, heterosynaptic calcium and
    overflowing fork stacks leave their values in the shared array; a different
    model advanced next must still equal pa_advance bit for bit."""
    dirty = [(W.recurrent_stc_morpho(n_exc=64, n_inh=16, d_p=1.0), E.FLAG_WIDE_ALL),
             (hca_tree_net(), 0),
             (tiny_tree_net(n_cells=70), 0)]
    for net, flags in dirty:
        m = E.Model(net, flags=flags)
        m.advance_noalloc(300 * net.dt)
        m.sync()
    assert E.Model(dirty[0][0], flags=E.FLAG_WIDE_ALL).info().n_wide > 0
    for precision in (E.PA_FP64, E.PA_MIXED):
        net = tiny_tree_net(n_cells=45, seed=11)
        ref = E.Model(net, precision=precision)
        new = E.Model(net, precision=precision)
        ref.advance(500 * net.dt)
        new.advance_noalloc(500 * net.dt)
        assert_same(ref, new)


def test_noalloc_allocates_no_device_memory():
    """Device memory is unchanged across calls after the first one (the first call
    on a GPU looks the array's address up, and with lazy module loading the
    driver reserves the array then)."""
    import torch
    net = small_net()
    m = E.Model(net, precision=E.PA_MIXED)
    m.advance_noalloc(10 * net.dt)
    m.sync()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for j in range(1, 6):
        m.advance_noalloc((10 + 97 * j) * net.dt)
    m.sync()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_refuses_models_beyond_its_scratch():
    # 2,097,152 padded CVs is the limit: 70,000 cells of 31 CVs exceed it
    b = W._Builder(0.1, 1, "big")
    pas = b.mech(W.PAS, W.pas_params())
    m = b.morph(W.ball_and_stick(20.0, 300.0, 1.0, 30))
    b.cells_add(70_000, m, pas, pas)
    net = b.build()
    model = E.Model(net)
    assert model.info().n_padded_cv > 2_097_152
    with pytest.raises(E.PaError) as ei:
        model.advance_noalloc(1.0)
    assert ei.value.code == -1 and "at most" in str(ei.value)
    model.advance(1.0)  # the allocating path still works


def test_noalloc_refuses_replay():
    net = small_net()
    model = E.Model(net)
    model.set_replay(np.array([0], np.int32), np.array([5], np.int64))
    with pytest.raises(E.PaError) as ei:
        model.advance_noalloc(1.0)
    assert ei.value.code == -6
