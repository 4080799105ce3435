"""Failure detection on the device without a GPU fault: the epoch kernel's
bounded waits for its staged rows are made to run out on purpose (a poll
limit of one non-blocking test, far shorter than a bulk copy's latency).  The
kernel must stop stepping, let every copy it issued land, return, and the host
must report PA_ERR_TIMEOUT at the next pa_sync -- with the CUDA context still
usable: the same model, its limit restored, and a fresh model both run again,
the fresh one bit-identical to the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2411_16445_b300 import engine as E

from _nets import tiny_tree_net

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("graphs", [False, True])
def test_wait_timeout_is_reported_and_the_context_stays_usable(graphs):
    net = tiny_tree_net(n_cells=70)
    flags = 0 if graphs else E.FLAG_NO_GRAPHS
    m = E.Model(net, precision=E.PA_FP64, flags=flags)
    m.advance(2 * m.info().epoch_steps * net.dt)
    m.sync()
    m.set_wait_limit(1)
    m.advance(10 * m.info().epoch_steps * net.dt)
    with pytest.raises(E.PaError) as ei:
        m.sync()
    assert ei.value.code == -4 and "wait" in str(ei.value)
    # the flag was consumed: the model runs on with the default limit (its
    # state is invalid after the timeout, so only the absence of errors counts)
    m.set_wait_limit(0)
    m.advance(14 * m.info().epoch_steps * net.dt)
    m.sync()
    # a fresh model on the same context is correct, bit for bit
    o = O.Oracle(net)
    o.run(800)
    f = E.Model(net, precision=E.PA_FP64, flags=flags)
    f.advance(800 * net.dt)
    f.sync()
    assert np.array_equal(o.v(), f.read_state(E.FIELD_V))
    assert np.array_equal(o.spikes()[1], f.read_spikes()[1])
