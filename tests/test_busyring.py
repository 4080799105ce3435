"""The busyring workload (Sec. "Runtime and memory benchmarking with large-scale
networks", Tables 7-9): structure against the paper's printed counts, and the
ring's spike circulating at 1 / (k t_delay) in the oracle."""
import numpy as np
import pytest

from paper_2411_16445_b300 import workloads as W


@pytest.mark.parametrize("depth,per_cell", [(0, 1.0), (2, 46116 / 1024), (10, 1672700 / 1024)])
def test_simple_branchy_matches_table8_compartment_counts(depth, per_cell):
    rng = np.random.default_rng(3)
    n = [W.simple_branchy(rng, depth).n_cv for _ in range(3000 if depth < 10 else 1500)]
    # Table 8: 1024 cells have 1024, 46116 and 1672700 compartments at depth 0, 2, 10
    assert abs(np.mean(n) - per_cell) <= 0.03 * per_cell
    m = W.simple_branchy(rng, depth)
    assert np.all(m.parent[1:] < np.arange(1, m.n_cv)) and m.region[0] == 0


def test_busyring_structure():
    net = W.busyring(n_cells=64, depth=2, s=1000)
    # 1.03M synapses for 1024 cells in Table 8: s random + 1 ring synapse per cell
    assert net.n_conn == 64 * 1001
    ring = net.conn_weight > 0
    assert ring.sum() == 64 and np.all(net.conn_cv[ring] == 0)
    assert np.all((net.conn_dst[ring] // 4) == (net.conn_src[ring] // 4))
    assert np.all(net.conn_delay == 5.0) and np.all(net.conn_weight[~ring] == 0.0)
    assert np.all(net.conn_cv < net.cell_ncv()[net.conn_dst])


@pytest.mark.parametrize("stdp", [False, True])
def test_ring_spike_circulates_in_the_oracle(stdp):
    import oracle as O
    net = W.busyring(n_cells=8, depth=2, s=10, stdp=stdp)
    o = O.Oracle(net)
    o.run(8000)                                # 200 ms at 0.025 ms
    g, _, t = o.spikes()
    # each cell fires once per lap: 1 / (4 x 5 ms) = 50 Hz, 10 spikes in 200 ms
    assert np.array_equal(np.bincount(g, minlength=8), np.full(8, 10))
    t0 = np.array([t[g == c][0] for c in range(4)])
    assert np.all(np.abs(np.diff(t0) - 5.0) < 0.2)
