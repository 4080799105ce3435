"""The bounds-checked build (libplasticarbor_checked.so, compiled with
-DPA_CHECKED): every global index of the time-step kernels and every bulk
copy's row range is checked against its array; a violation sets an error bit
that pa_sync reports instead of the access being made.  The small parity
cases run on it in a subprocess (the library is chosen with PA_LIBRARY before
the binding loads) -- narrow and wide bins, trees with fork stacks, several
synapse streams, partial epochs, heterosynaptic calcium, open-loop replay in
mixed precision and a batch -- with no violation and the FP64 results still
bit-identical to the oracle."""
import os
import subprocess
import sys

import pytest

from paper_2411_16445_b300 import build_lib

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
import oracle as O
from paper_2411_16445_b300 import engine as E
from paper_2411_16445_b300 import workloads as W
from _nets import edge_net, hca_tree_net, tiny_tree_net
assert E.LIB_PATH.endswith("libplasticarbor_checked.so")

def exact(net, steps, flags=0):
    o = O.Oracle(net); o.run(steps)
    m = E.Model(net, precision=E.PA_FP64, flags=flags)
    m.advance(steps * net.dt); m.sync()
    assert np.array_equal(o.v(), m.read_state(E.FIELD_V))
    assert np.array_equal(o.spikes()[1], m.read_spikes()[1])

exact(tiny_tree_net(), 1000)
exact(tiny_tree_net(n_cells=40), 600, E.FLAG_WIDE_ALL)
exact(edge_net(), 1001)
exact(hca_tree_net(), 800)
net = W.recurrent_stc(n_exc=80, n_inh=20, p=0.1, w_bg=3e-3, bg_rate=20.0)
ref = O.Oracle(net); ref.run(800); g, s, _ = ref.spikes()
m = E.Model(net, precision=E.PA_MIXED); m.set_replay(g, s); m.advance(800 * net.dt); m.sync()
b = E.Batch()
ms = [E.Model(W.serving_job(n, n % 2 == 0, 300.0, 1.0, n, dt=0.2), precision=E.PA_MIXED,
              flags=E.FLAG_NARROW_ONLY) for n in (3, 40, 200)]
for x in ms: b.add(x)
b.advance_epochs(12)
for x in ms: x.sync()
print("checked build: no violations")
'''


def test_small_parity_cases_on_the_checked_build():
    lib = build_lib.build(checked=True)
    env = dict(os.environ, PA_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT.replace("ROOT", repr(ROOT))], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "no violations" in r.stdout
