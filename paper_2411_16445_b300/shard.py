"""One network sharded over several GPUs: the cell partition, each rank's
network, and the per-epoch exchange of spikes.

The paper runs Arbor with one MPI rank per GPU (Sec. "Runtime and memory
benchmarking with large-scale networks"); it does not describe the exchange.
The design here follows from the loop itself:

  * cells are independent within a min-delay epoch of E steps (every
    connection's delay is at least E steps), so each rank advances its own
    cells through a whole epoch without communication;
  * rank r holds the cells of its part, every connection INTO those cells
    (Poisson trains keep their identity, so a cell sees the same drive as in
    the whole network), and one passive one-CV stand-in ("stub") per remote
    presynaptic cell; stubs never spike on their own;
  * after each epoch the ranks all-gather the epoch's spikes {gid, step}; each
    rank hands the spikes of remote cells that it holds stubs for to its
    model (pa_inject_spikes), which routes them through its own connection
    table exactly like local spikes.  Local spikes are routed locally by the
    model itself.

Every synapse sees the same events in the same steps as in the whole network,
and a cell's synapses keep their canonical order, so the sharded run equals
the single-model run bit for bit in FP64 (tested with the oracle on two gloo
ranks, and with two shard models on one GPU).  Plasticity noise is keyed by
the connection index within a model, so noisy models are not sharded.

Nothing here computes any of the method's arithmetic: it only builds
descriptors and moves spike lists.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, List, Sequence

import numpy as np

from . import workloads as W


def epoch_steps(net: W.Network, max_epoch_steps: int = 64) -> int:
    """The min-delay epoch E: the smallest delay, in steps, of any connection
    between cells (at least 1, at most max_epoch_steps)."""
    rec = net.conn_src >= 0
    if not np.any(rec):
        return max_epoch_steps
    d = np.maximum(1, np.rint(net.conn_delay[rec] / net.dt).astype(np.int64))
    return int(min(int(d.min()), max_epoch_steps))


def partition(net: W.Network, n_ranks: int) -> List[np.ndarray]:
    """Contiguous gid ranges with about equal work (CVs plus synapses into the
    cell), one per rank."""
    work = net.cell_ncv().astype(np.float64)
    work += np.bincount(net.conn_dst, minlength=net.n_cells)
    cum = np.cumsum(work)
    bounds = [0]
    for r in range(1, n_ranks):
        bounds.append(int(np.searchsorted(cum, cum[-1] * r / n_ranks)))
    bounds.append(net.n_cells)
    return [np.arange(bounds[r], bounds[r + 1], dtype=np.int64) for r in range(n_ranks)]


@dataclass
class Shard:
    net: W.Network          # the rank's model: own cells first, then the stubs
    own: np.ndarray         # global gids of the own cells (local gid i = own[i])
    stubs: np.ndarray       # global gids of the remote presynaptic cells (local n_own + j)
    local: np.ndarray       # [n_cells of the whole network] local gid, -1 if absent
    conn: np.ndarray        # indices (in the whole network) of the shard's connections


def shard_network(net: W.Network, own: Sequence[int]) -> Shard:
    """The network of one rank: the cells `own`, every connection into them in
    the whole network's order, and a stub for every remote presynaptic cell."""
    own = np.asarray(sorted(set(int(c) for c in own)), dtype=np.int64)
    conn = np.nonzero(np.isin(net.conn_dst, own))[0]
    src = net.conn_src[conn]
    stubs = np.setdiff1d(np.unique(src[src >= 0]), own)
    local = np.full(net.n_cells, -1, np.int64)
    local[own] = np.arange(len(own))
    local[stubs] = len(own) + np.arange(len(stubs))
    b = W._Builder(net.dt, net.seed, net.name + "_shard")
    for k, p in zip(net.mech_kind, net.mech_params):
        b.mech(int(k), p)
    stub_pas = b.mech(W.PAS, W.pas_params(3e-4, -65.0))
    morph_ids = {}
    for c in own:
        m = int(net.cell_morph[c])
        if m not in morph_ids:
            morph_ids[m] = b.morph(net.morphs[m])
        b.cells_add(1, morph_ids[m], int(net.cell_soma_mech[c]), int(net.cell_dend_mech[c]),
                    cm=net.cell_cm[c], ra=net.cell_ra[c], istep=net.cell_istep[c],
                    ton=net.cell_ton[c], toff=net.cell_toff[c], vinit=net.cell_vinit[c],
                    thresh=net.cell_thresh[c])
    if len(stubs):
        b.cells_add(len(stubs), b.morph(W.soma_only(10.0)), stub_pas, stub_pas, thresh=1e9)
    new_src = np.where(src >= 0, local[np.maximum(src, 0)], -1)
    b.connect(new_src, local[net.conn_dst[conn]], net.conn_cv[conn], net.conn_mech[conn],
              net.conn_weight[conn], delay=net.conn_delay[conn], rate=net.conn_rate[conn])
    sub = b.build()
    pid = net.conn_pid[conn].copy()
    pid[pid < 0] = conn[pid < 0]        # a Poisson train keeps its whole-network identity
    sub.conn_pid = pid.astype(np.int64)
    return Shard(sub, own, stubs, local, conn)


class ShardedRun:
    """Drives one rank's model epoch by epoch and exchanges the spikes.

    sim: the rank's model with advance_steps(n), read_spikes() -> (gid, step, t)
         of the spikes since the last call (local gids), and
         inject_spikes(gid, step) (local gids) -- an engine Model does;
    allgather: list of every rank's object, given this rank's (e.g.
         torch.distributed.all_gather_object around a list).
    """

    def __init__(self, shard: Shard, sim, E: int, allgather: Callable[[object], list]):
        self.shard, self.sim, self.E, self.allgather = shard, sim, E, allgather
        self.spikes = []                     # (global gid, step, t) of own cells

    def advance_epochs(self, n: int) -> None:
        own, local, n_own = self.shard.own, self.shard.local, len(self.shard.own)
        for _ in range(n):
            self.sim.advance_steps(self.E)
            g, s, t = self.sim.read_spikes()
            keep = g < n_own                 # stubs never spike; be explicit anyway
            gg = own[g[keep]]
            self.spikes.append((gg, s[keep], t[keep]))
            remote_g, remote_s = [], []
            for r, (og, os_) in enumerate(self.allgather((gg, s[keep]))):
                og = np.asarray(og, np.int64)
                if og.size == 0:
                    continue
                lg = local[og]
                sel = lg >= n_own            # remote cells this rank holds stubs for
                remote_g.append(lg[sel])
                remote_s.append(np.asarray(os_, np.int64)[sel])
            if remote_g:
                rg, rs = np.concatenate(remote_g), np.concatenate(remote_s)
                if rg.size:
                    order = np.lexsort((rg, rs))
                    self.sim.inject_spikes(rg[order].astype(np.int32), rs[order])

    def own_spikes(self):
        """(global gid, step, t) of this rank's cells, sorted by (step, gid)."""
        if not self.spikes:
            return (np.zeros(0, np.int64),) * 2 + (np.zeros(0),)
        g = np.concatenate([x[0] for x in self.spikes])
        s = np.concatenate([x[1] for x in self.spikes])
        t = np.concatenate([x[2] for x in self.spikes])
        o = np.lexsort((g, s))
        return g[o], s[o], t[o]


def run_local_shards(net: W.Network, n_ranks: int, make_sim: Callable[[Shard, int], object],
                     n_epochs: int, max_epoch_steps: int = 64):
    """All ranks' shards in one process, stepped in lock-step (the exchange as an
    in-process all-gather): the sharded design on one device or on the host.
    make_sim(shard, E) builds a rank's model.  Returns the shards and runs."""
    E = epoch_steps(net, max_epoch_steps)
    shards = [shard_network(net, own) for own in partition(net, n_ranks)]
    sims = [make_sim(sh, E) for sh in shards]
    box = {}

    def gather_for(r):
        def ag(obj):
            box[r] = obj
            return [box[q] for q in range(n_ranks)]
        return ag

    runs = [ShardedRun(sh, sim, E, gather_for(r)) for r, (sh, sim) in enumerate(zip(shards, sims))]
    for _ in range(n_epochs):
        # every rank advances its epoch, then all exchange (two phases)
        outs = []
        for r, run in enumerate(runs):
            run.sim.advance_steps(E)
            g, s, t = run.sim.read_spikes()
            n_own = len(run.shard.own)
            keep = g < n_own
            gg = run.shard.own[g[keep]]
            run.spikes.append((gg, s[keep], t[keep]))
            outs.append((gg, s[keep]))
        for r, run in enumerate(runs):
            local, n_own = run.shard.local, len(run.shard.own)
            rg, rs = [], []
            for og, os_ in outs:
                lg = local[og]
                sel = lg >= n_own
                rg.append(lg[sel])
                rs.append(np.asarray(os_, np.int64)[sel])
            rg, rs = np.concatenate(rg), np.concatenate(rs)
            if rg.size:
                order = np.lexsort((rg, rs))
                run.sim.inject_spikes(rg[order].astype(np.int32), rs[order])
    return shards, runs
