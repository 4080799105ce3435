"""pa_advance_noalloc: advancing a model without any GPU allocation during the call.

It is meant for callers that must not allocate device memory while they run --
code whose allocations belong to another memory manager, or a real-time host
thread where an allocation could stall or fail.  Its epoch kernel takes the
Hines elimination scratch from one fixed device array of the library instead
of from the model.  These tests check, through the C-ABI, that two calls in a
row give the same results as pa_advance (bit-identical in FP64, within the
mixed-precision voltage tolerance otherwise), and that too-large models and
replay mode are refused with an error.  The file is named so that pytest
collects it last; it also passes when run alone in a fresh process."""
import numpy as np
import pytest

from paper_2411_16445_b300 import engine as E
from paper_2411_16445_b300 import workloads as W

pytestmark = pytest.mark.gpu


def small_net():
    return W.recurrent_stc(n_exc=80, n_inh=20, p=0.1, w_bg=3e-3, bg_rate=20.0)


@pytest.mark.parametrize("precision", [E.PA_FP64, E.PA_MIXED])
def test_noalloc_matches_advance_on_two_calls(precision):
    net = small_net()
    ref = E.Model(net, precision=precision)
    new = E.Model(net, precision=precision)
    tol = 0.0 if precision == E.PA_FP64 else 1e-2  # mV
    for t_end in (40 * net.dt * 7 + 3 * net.dt, 40 * net.dt * 19):  # partial, then whole epochs
        ref.advance(t_end)
        new.advance_noalloc(t_end)
        ref.sync()
        new.sync()
        v_ref, v_new = ref.read_state(E.FIELD_V), new.read_state(E.FIELD_V)
        assert np.max(np.abs(v_ref - v_new)) <= tol
        g_ref, s_ref, _ = ref.read_spikes()
        g_new, s_new, _ = new.read_spikes()
        if precision == E.PA_FP64:
            assert np.array_equal(g_ref, g_new) and np.array_equal(s_ref, s_new)
            assert np.array_equal(ref.read_weights(), new.read_weights())
        else:
            assert len(g_ref) == len(g_new)


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
