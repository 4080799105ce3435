"""Signed zeros through the specialisation for reversal potentials of +0.

When every synapse stream has E = +0 the kernels form g E as the zero of g's
sign and skip the addition of the per-CV g E sum in the row assembly; the one
case where adding that signed zero changes a value (a right-hand side of -0
plus a +0 sum gives +0) takes a separate path.  These passive cells start at
V = -0 with a leak reversal of -0, so every dendritic right-hand side of the
first step is exactly -0 and the oracle's voltages become +0; later, a current
step and the Poisson drive move them off zero.  Voltages are compared bit for
bit (so -0 and +0 differ), in both cell bins, with E = +0 (specialised
kernels) and E = -0 (general kernels)."""
import numpy as np
import pytest

import oracle as O
from paper_2411_16445_b300 import engine as E
from paper_2411_16445_b300 import workloads as W

pytestmark = pytest.mark.gpu


def signed_zero_net(e_syn, n_cells=40, seed=3, dt=0.025):
    b = W._Builder(dt, seed, "signed_zero")
    rng = np.random.default_rng(seed)
    pas = b.mech(W.PAS, W.pas_params(3e-5, -0.0))
    syn = b.mech(W.EXPSYN, W.expsyn_params(2.0, e_syn))
    sizes = rng.integers(10, 61, n_cells)
    for c in range(n_cells):
        m = b.morph(W.random_binary_tree(rng, int(sizes[c])))
        # half the cells get a current step from step 50 on
        b.cells_add(1, m, pas, pas, vinit=-0.0, thresh=1e9,
                    istep=0.05 if c % 2 else 0.0, ton=50 * dt, toff=1e9)
    cv = (rng.random(n_cells) * sizes).astype(int)
    b.connect(W.SRC_POISSON, np.arange(n_cells), cv, syn, 1e-3, rate=50.0)
    return b.build()


def bits(v):
    return np.ascontiguousarray(v, dtype=np.float64).view(np.uint64)


@pytest.mark.parametrize("flags", [0, E.FLAG_WIDE_ALL])
@pytest.mark.parametrize("e_syn", [0.0, -0.0])
def test_signed_zero_voltages_bit_identical(e_syn, flags):
    net = signed_zero_net(e_syn)
    for steps in (1, 400):
        o = O.Oracle(net)
        o.run(steps)
        m = E.Model(net, precision=E.PA_FP64, flags=flags)
        m.advance(steps * net.dt)
        m.sync()
        vo, vg = o.v(), m.read_state(E.FIELD_V)
        if steps == 1:
            # the case under test occurred: -0 right-hand sides resolved to +0
            assert np.all(bits(vo) == 0)
        else:
            assert np.count_nonzero(vo) > len(vo) // 4
        assert np.array_equal(bits(vo), bits(vg)), \
            f"{np.count_nonzero(bits(vo) != bits(vg))} voltages differ in their bits"
        m.close()
