"""Parity of the CUDA engine (called through the C-ABI) with the FP64 oracle.

Tolerances (from the engine's specification): FP64 voltages within 1e-9 V
(1e-6 mV), mixed precision within 1e-5 V (1e-2 mV); identical spike counts,
spike times within 1e-3 ms; plastic weights within 1e-6 relative; spike
indices and event routing bit-exact.  The FP64 path is built to reproduce the
oracle's arithmetic operation for operation, so most FP64 checks below also
record whether the results are bit-identical."""
import numpy as np
import pytest

import oracle as O
from paper_2411_16445_b300 import engine as E
from paper_2411_16445_b300 import workloads as W

from _nets import (caterpillar_net, compare, edge_net, extract, fork_net, hca_tree_net,
                   map_spikes, tiny_tree_net)

pytestmark = pytest.mark.gpu

V_TOL = {E.PA_FP64: 1e-6, E.PA_MIXED: 1e-2, E.PA_FP32: 0.5}   # mV
W_RTOL = {E.PA_FP64: 1e-6, E.PA_MIXED: 1e-6, E.PA_FP32: 1e-3}
T_TOL = 1e-3                                     # ms
# PA_FP32 (the opt-in form: conductances, calcium, HH and the plasticity
# increments in FP32) does not meet the engine's tolerances on networks; its
# measured errors against the oracle on these networks are up to 0.12 mV,
# 0.09 ms (at dt 0.2 ms) and 1e-4 relative on the early-phase weight, with
# identical spike counts.  Its tests hold it to a few times those: V within
# 0.5 mV, spike times within dt / 2, weights within 1e-3 relative.
T_TOL_FP32_FRAC_DT = 0.5
PRECISIONS = [E.PA_FP64, E.PA_MIXED, E.PA_FP32]

FIELDS = [(O.SYN_G, E.FIELD_G), (O.SYN_C, E.FIELD_C), (O.SYN_W, E.FIELD_W),
          (O.SYN_H, E.FIELD_H), (O.SYN_Z, E.FIELD_Z), (O.SYN_APRE, E.FIELD_APRE),
          (O.SYN_APOST, E.FIELD_APOST)]


def run_both(net, steps, precision, probes=(), chunks=1, max_epoch_steps=0, flags=0):
    o = O.Oracle(net, probes=probes)
    o.run(steps)
    m = E.Model(net, precision=precision, probes=probes, max_epoch_steps=max_epoch_steps,
                flags=flags)
    per = steps // chunks
    done = 0
    for c in range(chunks):
        n = per if c < chunks - 1 else steps - done
        m.advance((done + n) * net.dt)
        done += n
    m.sync()
    return o, m


def run_replay_both(net, steps, precision, chunks=1, flags=0):
    """Mixed precision on networks: both sides driven by the oracle's closed-loop
    spike list (open-loop replay), so no chaotic amplification of rounding."""
    ref = O.Oracle(net)
    ref.run(steps)
    gid, step, _ = ref.spikes()
    o = O.Oracle(net)
    o.set_replay(gid, step)
    o.run(steps)
    m = E.Model(net, precision=precision, flags=flags)
    m.set_replay(gid, step)
    per = steps // chunks
    done = 0
    for c in range(chunks):
        n = per if c < chunks - 1 else steps - done
        m.advance((done + n) * net.dt)
        done += n
    m.sync()
    return o, m


def check_state(o, m, precision, exact=False):
    vo, vg = o.v(), m.read_state(E.FIELD_V)
    dv = compare(vo, vg)
    assert dv <= V_TOL[precision], f"max |dV| = {dv} mV"
    if exact:
        assert np.array_equal(vo, vg), f"FP64 path not bit-identical (max |dV| {dv})"
    go, so, to = o.spikes()
    gg, sg, tg = m.read_spikes()
    assert len(go) == len(gg), f"spike counts {len(go)} vs {len(gg)}"
    if precision == E.PA_FP64:
        assert np.array_equal(go, gg) and np.array_equal(so, sg), "spike indices differ"
        assert compare(to, tg) <= T_TOL
    else:
        # per cell: same number of spikes, matched crossing times
        dt = m.dt
        worst = 0.0
        for c in np.unique(np.concatenate([go, gg])):
            a, b = np.sort(to[go == c]), np.sort(tg[gg == c])
            assert len(a) == len(b), f"cell {c}: {len(a)} vs {len(b)} spikes"
            if len(a):
                worst = max(worst, float(np.max(np.abs(a - b))))
        bound = T_TOL if precision == E.PA_MIXED else T_TOL_FP32_FRAC_DT * dt
        assert worst <= bound, f"spike time error {worst} ms"
        print(f"precision {precision}: max |dV| {compare(vo, vg):.3e} mV, "
              f"max spike-time error {worst:.3e} ms")
    wo = o.syn(O.SYN_WEIGHT_TOTAL)
    wg = m.read_weights()
    assert np.all(np.abs(wo - wg) <= W_RTOL[precision] * np.maximum(np.abs(wo), 1e-12) + 1e-15)
    if precision == E.PA_FP64:
        for fo, fg in FIELDS:
            a, b = o.syn(fo), m.read_state(fg)
            assert compare(a, b) <= 1e-12 * max(1.0, np.abs(a).max() if a.size else 1.0)
        assert compare(o.cell_p(), m.read_state(E.FIELD_PRP)) <= 1e-12
        assert compare(o.gates().reshape(-1), m.read_state(E.FIELD_GATES)) <= 1e-12
    return dv


@pytest.mark.parametrize("precision", PRECISIONS)
def test_single_neuron_full_second(precision):
    """The single-neuron workload over its full 1 s (40,000 steps): soma and synapse
    CV traces every step, spikes, calcium and the GB weight."""
    net = W.single_neuron()
    probes = [(0, 0), (0, 33), (0, 64)]
    o, m = run_both(net, 40000, precision, probes=probes, chunks=7)
    po, pg = o.probes(), m.read_probes(len(probes))
    assert po.shape == pg.shape
    d = compare(po, pg)
    assert d <= V_TOL[precision], f"probe max |dV| = {d} mV"
    if precision == E.PA_FP64:
        assert np.array_equal(po, pg)
    check_state(o, m, precision, exact=precision == E.PA_FP64)


def test_recurrent_stc_closed_loop_fp64():
    """100-cell recurrent tagging-and-capture network (4 groups, ragged last group),
    closed loop: bit-identical spike trains, voltages, weights, tags and PRP."""
    net = W.recurrent_stc(n_exc=80, n_inh=20, p=0.1, w_bg=3e-3, bg_rate=20.0)
    o, m = run_both(net, 2500, E.PA_FP64, chunks=3)
    check_state(o, m, E.PA_FP64, exact=True)


@pytest.mark.parametrize("precision", [E.PA_MIXED, E.PA_FP32])
def test_recurrent_stc_mixed_open_loop(precision):
    net = W.recurrent_stc(n_exc=80, n_inh=20, p=0.1, w_bg=3e-3, bg_rate=20.0)
    o, m = run_replay_both(net, 2500, precision, chunks=3)
    check_state(o, m, precision)


def test_tree_cells_fp64_bit_exact():
    """Random binary trees: Hines elimination with branch points (children applied in
    descending order through the scratch arrays) and STDP."""
    net = tiny_tree_net()
    o, m = run_both(net, 3000, E.PA_FP64, chunks=2)
    check_state(o, m, E.PA_FP64, exact=True)


@pytest.mark.parametrize("precision", [E.PA_MIXED, E.PA_FP32])
def test_tree_cells_mixed_open_loop(precision):
    net = tiny_tree_net()
    o, m = run_replay_both(net, 3000, precision, chunks=2)
    check_state(o, m, precision)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_edge_cases(precision):
    """One-CV cells, a cell without synapses, several synapses of different mechanisms
    on one CV, a zero-rate Poisson train, a non-DFS branching numbering, delays that
    are not multiples of the epoch, partial epochs (odd advance chunks)."""
    net = edge_net()
    if precision == E.PA_FP64:
        o, m = run_both(net, 3001, precision, chunks=5)
    else:
        o, m = run_replay_both(net, 3001, precision, chunks=5)
    check_state(o, m, precision, exact=precision == E.PA_FP64)


def soma_over_two_cvs_net(dt=0.025, seed=21):
    """Passive cells whose soma region covers CVs 0 and 1, beside HH cells of
    the usual shape: the mixed kernels cannot form these groups' leak E-term
    from C/dt and read it from memory instead."""
    b = W._Builder(dt, seed, "soma_over_two_cvs")
    rng = np.random.default_rng(seed)
    hh = b.mech(W.HH, W.hh_params())
    pas = b.mech(W.PAS, W.pas_params())
    syn = b.mech(W.EXPSYN, W.expsyn_params(3.0, 0.0))
    m2 = W.ball_and_stick(20.0, 200.0, 1.5, 8)
    m2.region[1] = 0
    two = b.morph(m2)
    one = b.morph(W.ball_and_stick(20.0, 200.0, 1.5, 8))
    b.cells_add(40, two, pas, pas, istep=0.05)
    b.cells_add(8, one, hh, pas, istep=0.3)
    n = b.n_cells
    b.connect(W.SRC_POISSON, np.arange(n), rng.integers(0, 9, n), syn, 4e-3, rate=60.0)
    return b.build()


@pytest.mark.parametrize("precision", PRECISIONS)
def test_soma_over_two_cvs(precision):
    """Groups without the formed leak E-term: the oracle (FP64 bit for bit, the
    other forms within their bounds), and the two cell bins bit-identical."""
    net = soma_over_two_cvs_net()
    if precision == E.PA_FP64:
        o, m = run_both(net, 2000, precision, chunks=3)
    else:
        o, m = run_replay_both(net, 2000, precision, chunks=3)
    check_state(o, m, precision, exact=precision == E.PA_FP64)
    m.close()
    probes = [(0, 0), (0, 1), (net.n_cells - 1, 4)]
    a, na = _bin_run(net, precision, E.FLAG_NARROW_ONLY, probes)
    b, nb = _bin_run(net, precision, E.FLAG_WIDE_ALL, probes)
    assert na == 0 and nb == net.n_cells
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_morphology_sweep_small_fp64():
    net = W.morphology_sweep(n_nets=3, cells_per_net=40)
    o, m = run_both(net, 600, E.PA_FP64, chunks=2)
    check_state(o, m, E.PA_FP64, exact=True)


def test_morphology_sweep_small_mixed_open_loop():
    """The batched morphology sweep runs in mixed precision: GB synapses on chains of
    5-65 CVs, open-loop against the oracle at the mixed tolerances."""
    net = W.morphology_sweep(n_nets=3, cells_per_net=40)
    o, m = run_replay_both(net, 1500, E.PA_MIXED, chunks=2)
    check_state(o, m, E.PA_MIXED)
    for fo, fg in ((O.SYN_C, E.FIELD_C), (O.SYN_W, E.FIELD_W)):
        a, b = o.syn(fo), m.read_state(fg)
        assert np.all(np.abs(a - b) <= W_RTOL[E.PA_MIXED] * np.abs(a) + 1e-12), fg


def _large_stdp_small():
    """The large network's generator as the bench draws it (trees from a pool of
    shapes, 100-synapse fan-in, 1-5 ms delays, 2 Hz drive), at 1,024 cells."""
    return W.large_stdp(n_cells=1024, n_shapes=256)


# the launch configuration the bench times at full size: every cell in the
# thread-per-cell bin, kernel shape 0 (the autotuner's pick on that network)
BENCH_FLAGS = E.FLAG_NARROW_ONLY | E.flag_shape(0)


def test_large_stdp_generator_fp64_closed_loop():
    """Closed loop over 2,000 steps (50 ms; recurrent events and STDP updates),
    bit-identical to the oracle: voltages, spikes, weights and traces."""
    net = _large_stdp_small()
    o, m = run_both(net, 2000, E.PA_FP64, chunks=2, flags=BENCH_FLAGS)
    info = m.info()
    assert info.shape == 0 and info.n_wide == 0 and info.tree == 1
    assert len(o.spikes()[0]) > 50
    check_state(o, m, E.PA_FP64, exact=True)


def test_large_stdp_generator_mixed_open_loop():
    """The headline mixed path on the same network, open loop: V within 1e-5 V,
    per-cell spike times within 1e-3 ms, STDP w and both traces within 1e-6
    relative."""
    net = _large_stdp_small()
    o, m = run_replay_both(net, 2000, E.PA_MIXED, chunks=2, flags=BENCH_FLAGS)
    check_state(o, m, E.PA_MIXED)
    for fo, fg in ((O.SYN_W, E.FIELD_W), (O.SYN_APRE, E.FIELD_APRE),
                   (O.SYN_APOST, E.FIELD_APOST)):
        a, b = o.syn(fo), m.read_state(fg)
        assert np.all(np.abs(a - b) <= W_RTOL[E.PA_MIXED] * np.abs(a) + 1e-12), fg


def test_short_epochs_equal_long_epochs():
    """Routing once per epoch is exact for any epoch length <= the minimum delay."""
    net = tiny_tree_net(n_cells=40)
    m1 = E.Model(net, precision=E.PA_FP64, max_epoch_steps=3)
    m2 = E.Model(net, precision=E.PA_FP64)
    m1.advance(1200 * net.dt)
    m2.advance(1200 * net.dt)
    assert np.array_equal(m1.read_state(E.FIELD_V), m2.read_state(E.FIELD_V))
    assert np.array_equal(m1.read_spikes()[1], m2.read_spikes()[1])


@pytest.mark.parametrize("precision", [E.PA_FP64, E.PA_MIXED])
def test_open_loop_replay_stc(precision):
    """Open-loop replay: both sides are driven by the oracle's own spike list, so each
    cell's trajectory is compared without chaotic amplification."""
    net = W.recurrent_stc(n_exc=80, n_inh=20, p=0.1, w_bg=3e-3, bg_rate=20.0)
    ref = O.Oracle(net)
    ref.run(2000)
    gid, step, _ = ref.spikes()
    o = O.Oracle(net)
    o.set_replay(gid, step)
    o.run(2000)
    m = E.Model(net, precision=precision)
    m.set_replay(gid, step)
    m.advance(2000 * net.dt)
    dv = compare(o.v(), m.read_state(E.FIELD_V))
    assert dv <= V_TOL[precision]
    wo, wg = o.syn(O.SYN_WEIGHT_TOTAL), m.read_weights()
    assert np.all(np.abs(wo - wg) <= W_RTOL[precision] * np.abs(wo) + 1e-15)


def test_poisson_train_ids_shared():
    """Connections with the same poisson_id receive the same train."""
    b = W._Builder(0.1, 77, "pid")
    pas = b.mech(W.PAS, W.pas_params())
    e1 = b.mech(W.EXPSYN, W.expsyn_params(4.0, 0.0))
    m_ = b.morph(W.soma_only(20.0))
    b.cells_add(3, m_, pas, pas)
    b.connect(W.SRC_POISSON, [0, 1, 2], 0, e1, 1e-3, rate=50.0)
    net = b.build()
    net.conn_pid = np.array([5, 5, 6], np.int64)
    m = E.Model(net)
    m.advance(500.0)
    g = m.read_state(E.FIELD_G)
    assert g[0] == g[1] and g[0] != g[2]
    o = O.Oracle(net)
    o.run(5000)
    assert np.array_equal(o.syn(O.SYN_G), g)


def test_errors_are_reported_not_raised_on_device():
    net = W.single_neuron()
    with pytest.raises(E.PaError) as ei:
        bad = W.single_neuron()
        bad.conn_cv = np.array([999], np.int32)
        E.Model(bad)
    assert ei.value.code == -1
    m = E.Model(net)
    with pytest.raises(E.PaError):
        m.advance(0.0123)  # off the dt grid
    assert E.lib().pa_advance(m._h, 1.0, 0.05) == -1  # dt differs from the build-time dt
    # probe buffer overflow is reported as PA_ERR_CAPACITY, data kept up to capacity
    m2 = E.Model(net, probes=[(0, 0)], probe_capacity=100)
    m2.advance(200 * net.dt)
    with pytest.raises(E.PaError) as ei:
        m2.sync()
    assert ei.value.code == -5


@pytest.mark.parametrize("precision", PRECISIONS)
def test_every_kernel_shape_gives_identical_results(precision):
    """The compiled kernel shapes (TMA chunk sizes, warps per block, register budget)
    change scheduling only: every shape gives bit-identical results, and an
    autotuned model equals an untuned one."""
    net = tiny_tree_net(n_cells=70)
    ref = None
    for s in range(E.N_SHAPES):
        m = E.Model(net, precision=precision, flags=E.flag_shape(s))
        assert m.info().shape == s
        m.advance(800 * net.dt)
        v, sp = m.read_state(E.FIELD_V), m.read_spikes()[1]
        if ref is None:
            ref = (v, sp)
        assert np.array_equal(v, ref[0]) and np.array_equal(sp, ref[1])
    m = E.Model(net, precision=precision, flags=E.FLAG_AUTOTUNE)
    shape, ms = m.tuning()
    assert 0 <= shape < E.N_SHAPES and np.all(ms > 0) and ms[shape] == ms.min()
    m.advance(800 * net.dt)
    assert np.array_equal(m.read_state(E.FIELD_V), ref[0])


def test_trunk_first_and_side_first_numberings():
    """The same caterpillar tree numbered trunk-first (39 side branches wait for
    their parents at once in the elimination) and side-branch-first:
    bit-identical to the oracle."""
    net = caterpillar_net()
    o, m = run_both(net, 2000, E.PA_FP64, chunks=2)
    assert m.info().tree == 1
    check_state(o, m, E.PA_FP64, exact=True)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_graph_launches_equal_direct_launches(precision):
    """Whole epochs replayed from captured CUDA graphs (epoch taken from the
    device clock) give bit-identical voltages, probes, spikes and weights to
    direct launches, across partial epochs, probes, Poisson drive and delayed
    calcium targets."""
    net = edge_net()
    probes = [(3, 0), (5, 4), (6, 2)]
    runs = []
    for flags in (E.FLAG_NO_GRAPHS, 0):
        m = E.Model(net, precision=precision, probes=probes, flags=flags, probe_capacity=1000)
        steps = 0
        for n in (7, 160, 1, 333, 96, 15):     # partial and whole epochs
            steps += n
            m.advance(steps * net.dt)
        m.sync()
        ks = m.kernel_stats()
        runs.append((m.read_state(E.FIELD_V), m.read_probes(len(probes)), m.read_spikes(),
                     m.read_weights(), ks.graph_launches))
        m.close()
    (va, pa, sa, wa, ga), (vb, pb, sb, wb, gb) = runs
    assert ga == 0 and gb > 0
    assert np.array_equal(va, vb) and np.array_equal(pa, pb) and np.array_equal(wa, wb)
    for x, y in zip(sa, sb):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("stdp", [False, True])
def test_busyring_fp64_bit_exact(stdp):
    """The busyring benchmark network (rings of 4 simple-branchy cells, zero-weight
    random connections, optionally STDP): FP64 bit-identical to the oracle over
    40 ms, with the ring's spike circulating."""
    net = W.busyring(n_cells=48, depth=2, s=100, stdp=stdp)
    o, m = run_both(net, 1600, E.PA_FP64, chunks=3)
    go, _, _ = o.spikes()
    assert len(go) == 48 * 2          # every cell fires once per 20 ms lap
    check_state(o, m, E.PA_FP64, exact=True)


def _bin_run(net, precision, flags, probes):
    m = E.Model(net, precision=precision, probes=probes, flags=flags, probe_capacity=4000)
    steps = 0
    for n in (13, 250, 400, 97):              # partial and whole epochs
        steps += n
        m.advance(steps * net.dt)
    m.sync()
    out = [m.read_state(E.FIELD_V), m.read_probes(len(probes)), m.read_weights(),
           m.read_state(E.FIELD_G), m.read_state(E.FIELD_GATES), m.read_state(E.FIELD_PRP)]
    out += list(m.read_spikes())
    n_wide = m.info().n_wide
    m.close()
    return out, n_wide


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("which", ["trees", "edge", "busyring_stdp", "recurrent_stc"])
def test_wide_bin_equals_narrow_bin(precision, which):
    """Cells on a whole warp (synapses 32 at a time with an ordered fold, the tree
    eliminated branch-parallel by levels) give bit-identical states, probes,
    spikes and weights to cells on one thread each."""
    net = {"trees": lambda: tiny_tree_net(n_cells=40),
           "edge": edge_net,
           "busyring_stdp": lambda: W.busyring(n_cells=24, depth=3, s=60, stdp=True),
           "recurrent_stc": lambda: W.recurrent_stc(n_exc=64, n_inh=16)}[which]()
    ncv = net.cell_ncv()
    mid = net.n_cells // 2
    probes = [(0, 0), (net.n_cells - 1, int(ncv[-1]) - 1), (mid, int(ncv[mid]) // 2)]
    a, na = _bin_run(net, precision, E.FLAG_NARROW_ONLY, probes)
    b, nb = _bin_run(net, precision, E.FLAG_WIDE_ALL, probes)
    assert na == 0 and nb == net.n_cells
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_wide_bin_fp64_matches_oracle_and_automatic_bins():
    """The wide bin against the oracle, bit for bit, on the edge cases (non-DFS
    numbering, several synapse kinds on one CV, point cells); the automatic rule
    puts small busyring networks on whole warps and keeps large networks narrow."""
    net = edge_net()
    o = O.Oracle(net)
    o.run(3001)
    m = E.Model(net, precision=E.PA_FP64, flags=E.FLAG_WIDE_ALL)
    for n in (1000, 2001, 3001):
        m.advance(n * net.dt)
    m.sync()
    check_state(o, m, E.PA_FP64, exact=True)
    # between one and four narrow warps per SM: only large branched sparse cells
    ring = W.busyring(n_cells=6000, depth=10, s=30, n_shapes=256)
    ncv = ring.cell_ncv()
    nsyn = np.bincount(ring.conn_dst, minlength=ring.n_cells)
    nbr = np.array([1 + int(np.sum(m.parent[1:] != np.arange(m.n_cv - 1))) for m in ring.morphs])
    want = (ncv >= 128) & (nbr[ring.cell_morph] >= 8) & (nsyn <= 2 * ncv)
    assert E.Model(ring, precision=E.PA_MIXED).info().n_wide == int(want.sum()) > 3000
    # below one narrow warp per SM, cells with 128+ CVs plus synapses are wide too
    dense = W.busyring(n_cells=64, depth=2, s=100)
    heavy = dense.cell_ncv() + np.bincount(dense.conn_dst, minlength=dense.n_cells) >= 128
    assert E.Model(dense, precision=E.PA_MIXED).info().n_wide == int(heavy.sum())
    assert E.Model(tiny_tree_net(n_cells=40), precision=E.PA_MIXED).info().n_wide == 0


@pytest.mark.parametrize("precision", [E.PA_FP64, E.PA_MIXED])
def test_plasticity_noise_single_neuron(precision):
    """Graupner-Brunel weight with noise (sigma_pl = 2.8248, Table 3) on the
    single-neuron workload: the deviates of both sides are the same
    counter-based draws through the same log/sin/cos, so FP64 is bit-identical
    and the mixed path stays within its tolerances."""
    net = W.single_neuron(sigma_pl=2.8248)
    steps = 8000
    if precision == E.PA_FP64:
        o, m = run_both(net, steps, precision, chunks=3)
    else:
        o, m = run_replay_both(net, steps, precision, chunks=3)
    det = O.Oracle(W.single_neuron())
    det.run(steps)
    assert not np.array_equal(det.syn(O.SYN_W), o.syn(O.SYN_W))   # the noise acted
    check_state(o, m, precision, exact=precision == E.PA_FP64)


def test_plasticity_noise_recurrent_stc_fp64_closed_loop():
    """Early-phase weights with noise (sigma_pl = 2.90436 mV, Table 5) in a small
    recurrent STC network, closed loop: FP64 bit-identical to the oracle, in
    both cell bins."""
    net = W.recurrent_stc(n_exc=96, n_inh=24, sigma_pl=2.90436)
    o, m = run_both(net, 2500, E.PA_FP64, chunks=2)
    check_state(o, m, E.PA_FP64, exact=True)
    mw = E.Model(net, precision=E.PA_FP64, flags=E.FLAG_WIDE_ALL)
    mw.advance(2500 * net.dt)
    assert np.array_equal(mw.read_state(E.FIELD_H), o.syn(O.SYN_H))
    assert np.array_equal(mw.read_state(E.FIELD_V), o.v())


def _ff_sequence(model_or_oracle, net, is_oracle):
    """advance 1000 steps, fast-forward 10 s in 50 long steps, advance 1000 steps"""
    m = model_or_oracle
    if is_oracle:
        m.run(1000)
        m.fast_forward(int(round(10000.0 / net.dt)), 50)
        m.run(1000)
    else:
        m.advance(1000 * net.dt)
        m.fast_forward(10000.0, 50)
        m.advance((2000 + int(round(10000.0 / net.dt))) * net.dt)
        m.sync()


@pytest.mark.parametrize("precision", [E.PA_FP64, E.PA_MIXED])
def test_fast_forward_matches_oracle(precision):
    """Fast-forward of the slow plasticity variables between two stretches of
    full simulation (the '8h-recall' pattern) on the recurrent STC network with
    noise, closed loop: FP64 bit-identical to the oracle."""
    net = W.recurrent_stc(n_exc=96, n_inh=24, sigma_pl=2.90436)
    o = O.Oracle(net)
    _ff_sequence(o, net, True)
    m = E.Model(net, precision=precision)
    _ff_sequence(m, net, False)
    if precision == E.PA_FP64:
        check_state(o, m, precision, exact=True)
    else:   # mixed: the state after the fast-forward, before chaos sets in
        assert compare(o.cell_p(), m.read_state(E.FIELD_PRP)) <= 1e-9
        assert compare(o.syn(O.SYN_Z), m.read_state(E.FIELD_Z)) <= 1e-9


def test_state_swap_into_a_new_model():
    """Save every state field of a model, build a new model of the same network,
    move its clock to the same step, write the state in: both continue
    bit-identically (the state-saving mechanism of the '8h-recall' paradigm)."""
    net = W.recurrent_stc(n_exc=96, n_inh=24, sigma_pl=2.90436)
    a = E.Model(net, precision=E.PA_FP64)
    a.advance(1500 * net.dt)
    a.fast_forward(5000.0, 10)        # no events in flight, no POST_EVENT due
    fields = [E.FIELD_V, E.FIELD_GATES, E.FIELD_PRP, E.FIELD_G, E.FIELD_C, E.FIELD_W,
              E.FIELD_H, E.FIELD_Z]
    saved = {f: a.read_state(f) for f in fields}
    b = E.Model(net, precision=E.PA_FP64)
    b.fast_forward(1500 * net.dt + 5000.0, 1)
    for f in fields:
        b.write_state(f, saved[f])
        assert np.array_equal(b.read_state(f), saved[f])
    t_end = (1500 + int(round(5000.0 / net.dt)) + 1200) * net.dt
    for m in (a, b):
        m.advance(t_end)
    assert np.array_equal(a.read_state(E.FIELD_V), b.read_state(E.FIELD_V))
    assert np.array_equal(a.read_state(E.FIELD_H), b.read_state(E.FIELD_H))
    k_swap = 1500 + int(round(5000.0 / net.dt))
    ga, sa, _ = a.read_spikes()
    gb, sb, _ = b.read_spikes()
    after = sa >= k_swap
    assert len(gb) > 0 and np.array_equal(ga[after], gb) and np.array_equal(sa[after], sb)


def _diffusion_net(large_dend=False):
    # D_p = 1 um2/ms and tau_p = 200 ms so that the field moves within the run
    return W.recurrent_stc_morpho(n_exc=80, n_inh=20, d_p=1.0, tau_p=200.0, w_ext=0.02,
                                  large_dend=large_dend)


def _tag(net, seed=3):
    """early-phase weights above theta_tag on a random half of the E->E synapses
    (so that S exceeds theta_pro and PRP is synthesised)"""
    rng = np.random.default_rng(seed)
    h = np.zeros(net.n_conn)
    stc = net.conn_mech == 4
    h[stc] = 4.20075 + np.where(rng.random(stc.sum()) < 0.5, rng.uniform(0.9, 1.5, stc.sum()), 0.0)
    return h


@pytest.mark.parametrize("large_dend", [False, True])
def test_prp_diffusion_fp64_bit_exact(large_dend):
    """PRP diffusing over multi-compartment STC cells (31 / 48 CVs, branched at
    the soma), closed loop: the PRP field per CV, tags, weights, voltages and
    spikes bit-identical to the oracle."""
    net = _diffusion_net(large_dend)
    h = _tag(net)
    o = O.Oracle(net)
    o.set_syn(O.SYN_H, h)
    o.run(2500)
    m = E.Model(net, precision=E.PA_FP64)
    m.write_state(E.FIELD_H, h)
    for k in (700, 1900, 2500):
        m.advance(k * net.dt)
    m.sync()
    check_state(o, m, E.PA_FP64, exact=True)
    po, pg = o.prp(), m.read_state(E.FIELD_PRP_CV)
    assert np.array_equal(po, pg)
    exc = po.reshape(-1)[: 80 * net.morphs[0].n_cv].reshape(80, -1)
    assert exc.max() > 0 and np.any(exc[:, 0] > 1.2 * exc[:, -1])   # a field, not a pool
    assert np.all(po[80 * net.morphs[0].n_cv:] == 0)               # no field elsewhere


def test_prp_diffusion_mixed_open_loop():
    net = _diffusion_net()
    h = _tag(net)
    ref = O.Oracle(net)
    ref.set_syn(O.SYN_H, h)
    ref.run(2500)
    gid, step, _ = ref.spikes()
    o = O.Oracle(net)
    o.set_syn(O.SYN_H, h)
    o.set_replay(gid, step)
    o.run(2500)
    m = E.Model(net, precision=E.PA_MIXED)
    m.write_state(E.FIELD_H, h)
    m.set_replay(gid, step)
    m.advance(2500 * net.dt)
    m.sync()
    check_state(o, m, E.PA_MIXED)
    po, pg = o.prp(), m.read_state(E.FIELD_PRP_CV)
    assert compare(po, pg) <= 1e-9 * max(1.0, po.max())


def test_prp_diffusion_state_io_bins_and_fast_forward():
    """The field written per CV or uniformly per cell, read back, fast-forwarded
    (long reaction and diffusion steps) and continued bit-identically to the
    oracle with the same writes, in the thread-per-cell bin and with every
    cell in the warp-per-cell bin."""
    net = _diffusion_net()
    ncv = net.n_cv
    rng = np.random.default_rng(9)
    field = rng.uniform(0.0, 3.0, ncv)
    per_cell = rng.uniform(0.0, 3.0, net.n_cells)
    o = O.Oracle(net)
    o.set_syn(O.SYN_H, _tag(net))
    o.set_prp(field)
    o.run(300)
    o.set_cell_p(per_cell)
    o.run(300)
    o.fast_forward(int(round(2000.0 / net.dt)), 8)
    o.run(300)
    k_end = 600 + int(round(2000.0 / net.dt)) + 300
    for flags in (0, E.FLAG_WIDE_ALL):
        m = E.Model(net, precision=E.PA_FP64, flags=flags)
        if flags:
            assert m.info().n_wide == net.n_cells
        m.write_state(E.FIELD_H, _tag(net))
        m.write_state(E.FIELD_PRP_CV, field)
        got = m.read_state(E.FIELD_PRP_CV)
        want = np.where(np.repeat(np.arange(net.n_cells) < 80, net.cell_ncv()), field, 0.0)
        assert np.array_equal(got, want)
        m.advance(300 * net.dt)
        m.write_state(E.FIELD_PRP, per_cell)
        m.advance(600 * net.dt)
        m.fast_forward(2000.0, 8)
        m.advance(k_end * net.dt)
        m.sync()
        check_state(o, m, E.PA_FP64, exact=True)
        assert np.array_equal(o.prp(), m.read_state(E.FIELD_PRP_CV))


@pytest.mark.parametrize("precision", PRECISIONS)
def test_fork_stacks_every_shape(precision):
    """Fork stacks of every depth (and the shape without them) on trees whose
    forks nest far beyond the stacks, forks with several other children and
    random binary trees: FP64 bit-identical to the oracle in every shape,
    mixed identical across shapes."""
    net = fork_net()
    steps = 1200
    o = O.Oracle(net)
    o.run(steps) if precision == E.PA_FP64 else None
    ref = None
    for s in range(E.N_SHAPES):
        m = E.Model(net, precision=precision, flags=E.flag_shape(s) | E.FLAG_NARROW_ONLY)
        assert m.info().tree == 1 and m.info().n_wide == 0
        m.advance(steps * net.dt)
        m.sync()
        v = m.read_state(E.FIELD_V)
        if precision == E.PA_FP64:
            check_state(o, m, precision, exact=True)
        if ref is None:
            ref = v
        assert np.array_equal(v, ref), f"shape {s} differs"


def _hca_check(o, m, exact):
    vo, vg = o.v(), m.read_state(E.FIELD_V)
    if exact:
        assert np.array_equal(vo, vg)
    else:
        # PA_MIXED solves the cable in float-float: voltages within its tolerance
        assert compare(vo, vg) <= V_TOL[E.PA_MIXED]
    pairs = [(o.ca(), m.read_state(E.FIELD_CA_CV)),
             (o.syn(O.SYN_C), m.read_state(E.FIELD_C)), (o.syn(O.SYN_W), m.read_state(E.FIELD_W))]
    for a, b in pairs:
        if exact:
            assert np.array_equal(a, b)
        else:
            assert compare(a, b) <= 1e-9 * max(1.0, np.abs(a).max())


@pytest.mark.parametrize("precision", [E.PA_FP64, E.PA_MIXED])
def test_heterosynaptic_calcium_dendrite(precision):
    """The Table 4 dendrite with four spines, two of them driven by a regular
    100 Hz train (replayed): injection currents, the calcium field per CV and
    the weights, FP64 bit-identical to the oracle."""
    net, (gid, step) = W.heterosyn_dendrite(n_spikes=10)
    o = O.Oracle(net)
    o.set_replay(gid, step)
    m = E.Model(net, precision=precision)
    m.set_replay(gid, step)
    for t in (60.0, 150.0, 400.0):
        k = int(round(t / net.dt))
        o.run(k - o.step_count())
        m.advance(k * net.dt)
        m.sync()
        _hca_check(o, m, exact=precision == E.PA_FP64)
    ca = o.ca()
    assert ca[80] > 0 and ca[82] > 0 and np.all(o.syn(O.SYN_W) != 0.5)


def test_heterosynaptic_calcium_trees_closed_loop():
    """HCA synapses on random trees of a small recurrent network (Poisson and
    network events), closed loop: FP64 bit-identical, and the model refuses a
    fast-forward."""
    net = hca_tree_net()
    o, m = run_both(net, 3000, E.PA_FP64, chunks=2)
    check_state(o, m, E.PA_FP64, exact=True)
    _hca_check(o, m, exact=True)
    assert o.ca().max() > 0
    with pytest.raises(E.PaError):
        m.fast_forward(100.0, 2)
