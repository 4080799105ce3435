"""Helpers shared by the parity tests: small networks that exercise every code path,
sub-network extraction for sampled checks of full-size runs, and comparisons."""
from __future__ import annotations

import numpy as np

from paper_2411_16445_b300 import workloads as W


def extract(net: W.Network, cells) -> tuple:
    """The sub-network of `cells` with every connection into them.  Presynaptic cells
    outside the sample become one-CV passive stubs: in open-loop replay only their
    spike times matter.  Poisson connections keep their train ids, so the extracted
    cells see exactly the drive they see in the full network.
    Returns (subnet, old->new gid map, original indices of the kept connections)."""
    cells = np.asarray(sorted(set(int(c) for c in cells)), dtype=np.int64)
    keep = np.nonzero(np.isin(net.conn_dst, cells))[0]
    src = net.conn_src[keep]
    stubs = np.setdiff1d(np.unique(src[src >= 0]), cells)
    gmap = {int(g): i for i, g in enumerate(cells)}
    for j, g in enumerate(stubs):
        gmap[int(g)] = len(cells) + j
    b = W._Builder(net.dt, net.seed, net.name + "_sample")
    for k, p in zip(net.mech_kind, net.mech_params):
        b.mech(int(k), p)
    stub_pas = b.mech(W.PAS, W.pas_params(3e-4, -65.0))
    morph_ids = {}
    for c in cells:
        m = int(net.cell_morph[c])
        if m not in morph_ids:
            morph_ids[m] = b.morph(net.morphs[m])
        b.cells_add(1, morph_ids[m], int(net.cell_soma_mech[c]), int(net.cell_dend_mech[c]),
                    cm=net.cell_cm[c], ra=net.cell_ra[c], istep=net.cell_istep[c],
                    ton=net.cell_ton[c], toff=net.cell_toff[c], vinit=net.cell_vinit[c],
                    thresh=net.cell_thresh[c])
    if len(stubs):
        sm = b.morph(W.soma_only(10.0))
        b.cells_add(len(stubs), sm, stub_pas, stub_pas, thresh=1e9)
    new_src = np.array([gmap[int(s)] if s >= 0 else -1 for s in src], dtype=np.int64)
    new_dst = np.array([gmap[int(d)] for d in net.conn_dst[keep]], dtype=np.int64)
    b.connect(new_src, new_dst, net.conn_cv[keep], net.conn_mech[keep], net.conn_weight[keep],
              delay=net.conn_delay[keep], rate=net.conn_rate[keep])
    sub = b.build()
    pid = net.conn_pid[keep].copy()
    pid[pid < 0] = keep[pid < 0]
    sub.conn_pid = pid.astype(np.int64)
    return sub, gmap, keep


def map_spikes(gid, step, gmap):
    """Spikes of the full network restricted to the extracted cells, renumbered and
    sorted by (step, gid)."""
    sel = [(gmap[int(g)], int(s)) for g, s in zip(gid, step) if int(g) in gmap]
    sel.sort(key=lambda x: (x[1], x[0]))
    return (np.array([x[0] for x in sel], np.int32), np.array([x[1] for x in sel], np.int64))


def tiny_tree_net(n_cells=45, seed=5, dt=0.025, stdp=True):
    """Random binary trees (10-60 dendritic CVs), HH somata, STDP and static synapses,
    Poisson drive strong enough to make cells fire; n_cells not a multiple of 32."""
    b = W._Builder(dt, seed, "tiny_tree")
    rng = np.random.default_rng(seed)
    hh = b.mech(W.HH, W.hh_params())
    pas = b.mech(W.PAS, W.pas_params())
    syn = b.mech(W.STDP if stdp else W.EXPSYN,
                 W.stdp_params(w0=0.6) if stdp else W.expsyn_params())
    drive = b.mech(W.EXPSYN, W.expsyn_params(2.0, 0.0))
    sizes = rng.integers(10, 61, n_cells)
    for c in range(n_cells):
        m = b.morph(W.random_binary_tree(rng, int(sizes[c])))
        b.cells_add(1, m, hh, pas)
    n_conn = n_cells * 12
    src = rng.integers(0, n_cells, n_conn)
    dst = rng.integers(0, n_cells, n_conn)
    ok = src != dst
    src, dst = src[ok], dst[ok]
    cv = 1 + (rng.random(len(dst)) * sizes[dst]).astype(int)
    D = rng.integers(8, 40, len(dst))
    b.connect(src, dst, cv, syn, 2e-3, delay=D * dt)
    b.connect(W.SRC_POISSON, np.arange(n_cells), 0, drive, 0.08, rate=40.0)
    return b.build()


def edge_net(dt=0.1, seed=9):
    """Degenerate shapes: one-CV cells, a cell without synapses, a cell with several
    synapses on one CV, zero-rate Poisson drive, mixed synapse kinds on one cell,
    non-DFS tree numbering and a synapse on the root of a branching cell."""
    b = W._Builder(dt, seed, "edge")
    hh = b.mech(W.HH, W.hh_params())
    pas = b.mech(W.PAS, W.pas_params())
    e1 = b.mech(W.EXPSYN, W.expsyn_params(3.0, 0.0))
    e2 = b.mech(W.EXPSYN, W.expsyn_params(8.0, -80.0))
    gb = b.mech(W.GB, W.gb_params(t_c_delay=2.0, tau_w=5e3))
    stdp = b.mech(W.STDP, W.stdp_params(tau_pre=5.0, tau_post=7.0))
    m1 = b.morph(W.soma_only(18.0))
    m2 = b.morph(W.ball_and_stick(20.0, 150.0, 1.5, 5))
    # non-DFS numbering: 0 -> {1, 2}, 1 -> {3, 5}, 2 -> {4}
    par = np.array([-1, 0, 0, 1, 2, 1], np.int32)
    m3 = b.morph(W.Morphology(par, np.full(6, 15.0), np.array([16, 2, 2, 1, 1, 1.0]),
                              np.array([0, 1, 1, 1, 1, 1], np.int32)))
    b.cells_add(3, m1, hh, pas, istep=0.06)            # 0..2 point cells
    b.cells_add(2, m2, hh, pas, istep=0.0)             # 3, 4
    b.cells_add(2, m3, hh, pas, istep=0.3)             # 5, 6
    b.cells_add(1, m2, pas, pas)                       # 7: passive, no synapses at all
    b.connect(W.SRC_POISSON, 3, 2, e1, 5e-3, rate=80.0)
    b.connect(W.SRC_POISSON, 3, 2, e2, 1e-3, rate=30.0)
    b.connect(W.SRC_POISSON, 4, 0, gb, 4e-3, rate=60.0)
    b.connect(W.SRC_POISSON, 4, 0, e1, 4e-3, rate=0.0)
    b.connect([0, 1, 2, 5, 6, 0], [3, 4, 5, 6, 5, 4], [1, 3, 0, 4, 5, 2],
              [e1, gb, stdp, stdp, gb, e2], [3e-3, 2e-3, 4e-3, 4e-3, 3e-3, 2e-3],
              delay=[0.4, 1.0, 0.3, 2.2, 0.7, 6.3])
    return b.build()


def caterpillar_net(n_trunk=40, dt=0.025, seed=13):
    """Cells whose depth-first numbering visits the whole trunk before any side
    branch (soma, trunk 1..n_trunk, then side CVs n_trunk+1.. of trunk nodes
    n_trunk..1), so that n_trunk - 1 side branches wait for their parents at
    once in the elimination, plus cells of the same tree numbered
    side-branch-first."""
    b = W._Builder(dt, seed, "caterpillar")
    hh = b.mech(W.HH, W.hh_params())
    pas = b.mech(W.PAS, W.pas_params())
    syn = b.mech(W.EXPSYN, W.expsyn_params(3.0, 0.0))
    n = 1 + 2 * n_trunk
    par = np.empty(n, np.int32)
    par[0] = -1
    par[1:n_trunk + 1] = np.arange(0, n_trunk)
    par[n_trunk + 1:] = np.arange(n_trunk, 0, -1)          # side CV of trunk node t
    diam = np.r_[18.0, np.full(n_trunk, 2.0), np.full(n_trunk, 0.8)]
    region = np.r_[0, np.ones(n - 1, np.int32)].astype(np.int32)
    m_deep = b.morph(W.Morphology(par, np.full(n, 12.0), diam, region))
    # side-branch-first: trunk node t = 2t-1, its side CV 2t
    par2 = np.empty(n, np.int32)
    par2[0] = -1
    for t in range(1, n_trunk + 1):
        par2[2 * t - 1] = 0 if t == 1 else 2 * t - 3
        par2[2 * t] = 2 * t - 1
    diam2 = np.r_[18.0, np.tile([2.0, 0.8], n_trunk)]
    m_flat = b.morph(W.Morphology(par2, np.full(n, 12.0), diam2, region))
    b.cells_add(3, m_deep, hh, pas, istep=0.25)
    b.cells_add(2, m_flat, hh, pas, istep=0.25)
    rng = np.random.default_rng(seed)
    b.connect(W.SRC_POISSON, np.arange(5), rng.integers(1, n, 5), syn, 4e-3, rate=60.0)
    return b.build()


def fork_net(dt=0.025, seed=21):
    """Trees for the fork stacks: a caterpillar numbered trunk-first (39 forks
    pending at once, far beyond the stacks' depth), the same with its side CVs
    in trunk order (not nested), a star (a soma with five dendrites, and one
    dendrite node with three children: forks with several other children) and
    random binary trees (many short branches)."""
    b = W._Builder(dt, seed, "forks")
    rng = np.random.default_rng(seed)
    hh = b.mech(W.HH, W.hh_params())
    pas = b.mech(W.PAS, W.pas_params())
    syn = b.mech(W.EXPSYN, W.expsyn_params(3.0, 0.0))
    n_trunk = 40
    n = 1 + 2 * n_trunk
    par = np.empty(n, np.int32)
    par[0] = -1
    par[1:n_trunk + 1] = np.arange(0, n_trunk)
    par[n_trunk + 1:] = np.arange(n_trunk, 0, -1)
    cat = W.Morphology(par, np.full(n, 12.0), np.r_[18.0, np.full(n - 1, 1.5)],
                       np.r_[0, np.ones(n - 1)].astype(np.int32))
    # star: soma 0; dendrites start at 1, 6, 11, 16, 21 (5 CVs each); node 13 has
    # children 14 (first), 26 and 27 (two other children)
    spar = [-1]
    for d in range(5):
        start = len(spar)
        spar += [0] + list(range(start, start + 4))
    spar += [13, 13]
    spar = np.asarray(spar, np.int32)
    star = W.Morphology(spar, np.full(len(spar), 10.0), np.r_[16.0, np.full(len(spar) - 1, 1.2)],
                        np.r_[0, np.ones(len(spar) - 1)].astype(np.int32))
    # the same caterpillar with its side CVs numbered in trunk order: the pushes
    # and pops of the fork stacks would not nest (the kernel keeps the lists)
    par2 = par.copy()
    par2[n_trunk + 1:] = np.arange(1, n_trunk + 1)
    cat2 = W.Morphology(par2, np.full(n, 12.0), np.r_[18.0, np.full(n - 1, 1.5)],
                        np.r_[0, np.ones(n - 1)].astype(np.int32))
    m_cat, m_star, m_cat2 = b.morph(cat), b.morph(star), b.morph(cat2)
    b.cells_add(9, m_cat, hh, pas, istep=0.3)
    b.cells_add(9, m_star, hh, pas, istep=0.25)
    b.cells_add(5, m_cat2, hh, pas, istep=0.3)
    for _ in range(30):
        m = b.morph(W.random_binary_tree(rng, int(rng.integers(20, 120))))
        b.cells_add(1, m, hh, pas, istep=0.2)
    ncv = b.build().cell_ncv()
    dst = np.repeat(np.arange(len(ncv)), 3)
    cv = (rng.random(len(dst)) * ncv[dst]).astype(int)
    b.connect(W.SRC_POISSON, dst, cv, syn, 3e-3, rate=50.0)
    return b.build()


def compare(a, b):
    a, b = np.asarray(a), np.asarray(b)
    assert a.shape == b.shape, (a.shape, b.shape)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)))


def hca_tree_net():
    """HCA synapses on random trees of a small recurrent network (40 HH cells of
    8-50 dendritic CVs, 300 network and 60 Poisson HCA synapses, somatic Poisson
    drive)."""
    dt = 0.025
    b = W._Builder(dt, 31, "hca_trees")
    rng = np.random.default_rng(31)
    hh = b.mech(W.HH, W.hh_params())
    pas = b.mech(W.PAS, W.pas_params())
    drive = b.mech(W.EXPSYN, W.expsyn_params(2.0, 0.0))
    hca = b.mech(W.HCA, W.hca_params(d=0.5, tau_c=40.0, i0=6.0))
    sizes = rng.integers(8, 50, 40)
    for c in range(40):
        b.cells_add(1, b.morph(W.random_binary_tree(rng, int(sizes[c]))), hh, pas)
    b.connect(W.SRC_POISSON, np.arange(40), 0, drive, 0.08, rate=40.0)
    src = rng.integers(0, 40, 300)
    dst = rng.integers(0, 40, 300)
    cv = (rng.random(300) * (sizes[dst] + 1)).astype(int)
    b.connect(src, dst, cv, hca, 1.0, delay=1.0)
    b.connect(W.SRC_POISSON, dst[:60], cv[:60], hca, 1.0, rate=30.0)
    return b.build()
