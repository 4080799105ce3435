"""Seeded synthetic inputs: morphologies, cells, mechanism tables, connections.

This module only *describes* networks (shapes, parameter tables, random
connectivity).  It holds none of the simulated method's arithmetic, so both the
CUDA engine and the CPU oracle can be fed from it.  The workloads follow the
configurations the engine is measured on, with the paper's parameter tables
(Tables 3 and 5) and the readings listed in the design notes where the
configurations are silent.

Units: mV, ms, um, uS (weights), nA, S/cm2, uF/cm2, ohm cm.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Mechanism kinds (descriptor format shared by the engine's C-ABI and the oracle).
PAS, HH, EXPSYN, GB, STC, STDP, HCA = 1, 2, 10, 11, 12, 13, 14
SRC_POISSON = -1
NEVER = 1e300  # t_off meaning "never switched off"

MASTER_SEED = 20241125


def config_seed(name: str, master: int = MASTER_SEED) -> int:
    """Per-workload seed: an FNV-style integer hash of the workload name and the master seed."""
    h = master & 0xFFFFFFFFFFFFFFFF
    for ch in name.encode():
        h = ((h ^ ch) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


# --------------------------------------------------------------------------
# parameter tables
def hh_params(gnabar=0.12, gkbar=0.036, gl=3e-4, ena=50.0, ek=-77.0, el=-54.4):
    return np.array([gnabar, gkbar, gl, ena, ek, el])


def pas_params(g=3e-5, e=-54.4):
    return np.array([g, e])


def expsyn_params(tau=5.0, e=0.0):
    return np.array([tau, e])


def gb_params(tau=5.0, e=0.0, tau_c=20.0, c_pre=1.0, c_post=2.0, theta_p=1.3, theta_d=1.0,
              gamma_p=725.0, gamma_d=331.0, tau_w=346.0e3, w_star=0.5, t_c_delay=13.7, w0=0.0,
              sigma_pl=0.0):
    """Graupner-Brunel calcium rule (Eqs. weight_graupner_brunel, ca_model_graupner_brunel,
    plasticity_noise_1).  Defaults: the single-neuron workload's constants; w_star and
    t_c_delay from Table 3; sigma_pl = 0 (deterministic; Table 3 gives 2.8248)."""
    return np.array([tau, e, tau_c, c_pre, c_post, theta_p, theta_d, gamma_p, gamma_d, tau_w,
                     w_star, t_c_delay, w0, sigma_pl])


def stc_params(tau=5.0, e=0.0, tau_c=48.8, c_pre=0.6, c_post=0.1655, theta_p=3.0, theta_d=1.2,
               gamma_p=1645.6, gamma_d=313.1, tau_h=688.4e3, tau_z=3600.0e3, tau_p=3600.0e3,
               h0=4.20075, theta_tag=0.840149, theta_pro=2.10037, p_max=10.0, f_int=0.1,
               t_c_delay=18.8, sigma_pl=0.0, d_p=0.0):
    """Tagging-and-capture rule (Eqs. total_syn_weight .. prp_single_comp,
    plasticity_noise_2), Table 5 with the in-vivo calcium contributions used for
    networks; sigma_pl = 0 (deterministic; Table 5 gives 2.90436 mV).  d_p > 0
    [um2/ms] makes the PRP a concentration per CV that diffuses over the cell
    (Eq. diffusion; 1e-11 m2/s = 1e-2 um2/ms)."""
    p = [tau, e, tau_c, c_pre, c_post, theta_p, theta_d, gamma_p, gamma_d, tau_h,
         tau_z, tau_p, h0, theta_tag, theta_pro, p_max, f_int, t_c_delay, sigma_pl]
    if d_p > 0.0:
        p.append(d_p)
    return np.array(p)


def hca_params(i0=4.0, tau_i=1.0, gamma=0.11, gamma_p=90.0, gamma_d=0.01, theta_p=0.11,
               theta_d=0.05, w0=0.5, tau_c=100.0, d=0.22):
    """Heterosynaptic calcium rule (Eqs. ca_injection_current_spine,
    ca_diffusion_dendrite, heterosyn_weight; Table 4, Arbor's I0 = 4 pA):
    I0 [pA], tau_I [ms], gamma, gamma_p, gamma_d [1/s], theta_p, theta_d
    [umol/l], w0 (not in Table 4), tau_C [ms], D [um2/ms] (2.2e-10 m2/s)."""
    return np.array([i0, tau_i, gamma, gamma_p, gamma_d, theta_p, theta_d, w0, tau_c, d])


def stdp_params(tau=5.0, e=0.0, tau_pre=16.8, tau_post=33.7, a_pre=0.01, a_post=-0.012,
                w0=0.5, w_max=1.0):
    """Pair STDP (Eqs. stdp_ode_1-3); w dimensionless, conductance weight*clip(w, 0, w_max)."""
    return np.array([tau, e, tau_pre, tau_post, a_pre, a_post, w0, w_max])


# --------------------------------------------------------------------------
@dataclasses.dataclass
class Morphology:
    parent: np.ndarray   # int32, parent[0] = -1, parent[i] < i
    length: np.ndarray   # float64 um
    diam: np.ndarray     # float64 um
    region: np.ndarray   # int32: 0 soma, 1 dendrite

    @property
    def n_cv(self) -> int:
        return int(self.parent.shape[0])

    def is_chain(self) -> bool:
        return bool(np.all(self.parent[1:] == np.arange(self.n_cv - 1)))


@dataclasses.dataclass
class Network:
    dt: float
    seed: int
    mech_kind: np.ndarray                  # int32 [M]
    mech_params: List[np.ndarray]
    morphs: List[Morphology]
    cell_morph: np.ndarray                 # int32 [N]
    cell_soma_mech: np.ndarray
    cell_dend_mech: np.ndarray
    cell_cm: np.ndarray                    # float64 [N]
    cell_ra: np.ndarray
    cell_istep: np.ndarray
    cell_ton: np.ndarray
    cell_toff: np.ndarray
    cell_vinit: np.ndarray
    cell_thresh: np.ndarray
    conn_src: np.ndarray                   # int32 [C]
    conn_dst: np.ndarray
    conn_cv: np.ndarray
    conn_mech: np.ndarray
    conn_weight: np.ndarray                # float64 [C]
    conn_delay: np.ndarray
    conn_rate: np.ndarray
    conn_pid: Optional[np.ndarray] = None  # int64 Poisson train id (-1: connection index)
    name: str = "custom"

    def __post_init__(self):
        if self.conn_pid is None:
            self.conn_pid = np.full(self.conn_src.shape[0], -1, dtype=np.int64)

    @property
    def n_cells(self) -> int:
        return int(self.cell_morph.shape[0])

    @property
    def n_conn(self) -> int:
        return int(self.conn_src.shape[0])

    def cell_ncv(self) -> np.ndarray:
        sizes = np.array([m.n_cv for m in self.morphs], dtype=np.int64)
        return sizes[self.cell_morph]

    @property
    def n_cv(self) -> int:
        return int(self.cell_ncv().sum())

    def packed_morphs(self):
        ncv = np.array([m.n_cv for m in self.morphs], dtype=np.int32)
        off = np.zeros(len(self.morphs), dtype=np.int32)
        if len(self.morphs) > 1:
            off[1:] = np.cumsum(ncv[:-1])

        def cat(f, dt_):
            if not self.morphs:
                return np.zeros(0, dt_)
            return np.concatenate([getattr(m, f) for m in self.morphs]).astype(dt_)

        return (ncv, off, cat("parent", np.int32), cat("length", np.float64),
                cat("diam", np.float64), cat("region", np.int32))

    def packed_mechs(self):
        off = np.zeros(len(self.mech_params), dtype=np.int32)
        sizes = [len(p) for p in self.mech_params]
        if len(sizes) > 1:
            off[1:] = np.cumsum(sizes[:-1])
        params = (np.concatenate(self.mech_params).astype(np.float64)
                  if self.mech_params else np.zeros(0))
        return self.mech_kind.astype(np.int32), off, params


class _Builder:
    """Accumulates mechanisms, morphologies, cells and connections (numpy chunks)."""

    _CELL = (("morph", np.int32), ("soma", np.int32), ("dend", np.int32), ("cm", np.float64),
             ("ra", np.float64), ("istep", np.float64), ("ton", np.float64),
             ("toff", np.float64), ("vinit", np.float64), ("thresh", np.float64))
    _CONN = (("src", np.int32), ("dst", np.int32), ("cv", np.int32), ("mech", np.int32),
             ("w", np.float64), ("delay", np.float64), ("rate", np.float64))

    def __init__(self, dt: float, seed: int, name: str):
        self.dt, self.seed, self.name = dt, seed, name
        self.mk, self.mp, self.morphs = [], [], []
        self.cells = {k: [] for k, _ in self._CELL}
        self.conn = {k: [] for k, _ in self._CONN}
        self.n_cells = 0

    def mech(self, kind: int, params) -> int:
        self.mk.append(kind)
        self.mp.append(np.asarray(params, dtype=np.float64))
        return len(self.mk) - 1

    def morph(self, m: Morphology) -> int:
        self.morphs.append(m)
        return len(self.morphs) - 1

    def cells_add(self, n, morph, soma, dend, cm=1.0, ra=100.0, istep=0.0, ton=0.0, toff=NEVER,
                  vinit=-65.0, thresh=-10.0) -> np.ndarray:
        start = self.n_cells
        vals = dict(morph=morph, soma=soma, dend=dend, cm=cm, ra=ra, istep=istep, ton=ton,
                    toff=toff, vinit=vinit, thresh=thresh)
        for k, dt_ in self._CELL:
            self.cells[k].append(np.broadcast_to(np.asarray(vals[k], dtype=dt_), (n,)).copy())
        self.n_cells += n
        return np.arange(start, start + n)

    def connect(self, src, dst, cv, mech, w, delay=0.0, rate=0.0) -> None:
        n = len(np.atleast_1d(dst))
        vals = dict(src=src, dst=dst, cv=cv, mech=mech, w=w, delay=delay, rate=rate)
        for k, dt_ in self._CONN:
            self.conn[k].append(np.broadcast_to(np.asarray(vals[k], dtype=dt_), (n,)).copy())

    def build(self) -> Network:
        def cat(d, k, dt_):
            return np.concatenate(d[k]).astype(dt_) if d[k] else np.zeros(0, dt_)

        c = {k: cat(self.cells, k, t) for k, t in self._CELL}
        k = {kk: cat(self.conn, kk, t) for kk, t in self._CONN}
        return Network(
            dt=self.dt, seed=self.seed, mech_kind=np.asarray(self.mk, np.int32),
            mech_params=self.mp, morphs=self.morphs, cell_morph=c["morph"],
            cell_soma_mech=c["soma"], cell_dend_mech=c["dend"], cell_cm=c["cm"],
            cell_ra=c["ra"], cell_istep=c["istep"], cell_ton=c["ton"], cell_toff=c["toff"],
            cell_vinit=c["vinit"], cell_thresh=c["thresh"], conn_src=k["src"],
            conn_dst=k["dst"], conn_cv=k["cv"], conn_mech=k["mech"], conn_weight=k["w"],
            conn_delay=k["delay"], conn_rate=k["rate"], name=self.name)


# --------------------------------------------------------------------------
# morphologies
def ball_and_stick(soma_diam=20.0, dend_len=500.0, dend_diam=1.0, n_dend=64) -> Morphology:
    """Soma: one cylinder with length = diameter (lateral area of the sphere).
    Dendrite: n_dend equal cylinders in a chain from the soma."""
    n = 1 + n_dend
    parent = np.arange(-1, n - 1, dtype=np.int32)
    length = np.full(n, dend_len / max(n_dend, 1))
    diam = np.full(n, dend_diam)
    length[0], diam[0] = soma_diam, soma_diam
    region = np.ones(n, dtype=np.int32)
    region[0] = 0
    return Morphology(parent, length, diam, region)


def soma_only(diam=20.0) -> Morphology:
    return Morphology(np.array([-1], np.int32), np.array([diam]), np.array([diam]),
                      np.array([0], np.int32))


def random_binary_tree(rng: np.random.Generator, n_dend: int, soma_diam=20.0,
                       branch_len=(20.0, 100.0), max_cv_len=20.0, diam_root=2.0,
                       diam_tip=0.5) -> Morphology:
    """Random binary dendritic tree of exactly n_dend CVs on a soma CV.

    Grows branches from the soma by splitting a uniformly chosen open tip into
    two child branches; each branch has a length ~ U(branch_len) discretised
    into CVs of at most max_cv_len; growth stops at n_dend CVs (the last branch
    is truncated).  Diameters taper linearly with branch order from diam_root
    (order 0) to diam_tip (deepest order).  CVs are numbered depth-first so
    parent[i] < i."""
    branches = []  # (parent_branch, order, n_cv, cv_len)
    remaining = n_dend
    tips = []

    def new_branch(pb, order):
        nonlocal remaining
        L = rng.uniform(*branch_len)
        full = max(1, int(math.ceil(L / max_cv_len)))
        ncv = min(full, remaining)
        branches.append((pb, order, ncv, L / full))
        remaining -= ncv
        tips.append(len(branches) - 1)

    new_branch(-1, 0)
    while remaining > 0:
        t = tips.pop(int(rng.integers(len(tips))))
        new_branch(t, branches[t][1] + 1)
        if remaining > 0:
            new_branch(t, branches[t][1] + 1)
    max_order = max(b[1] for b in branches)
    children = [[] for _ in branches]
    for i, b in enumerate(branches):
        if b[0] >= 0:
            children[b[0]].append(i)
    parent, length, diam = [-1], [soma_diam], [soma_diam]
    stack = [(0, 0)]  # (branch, parent CV)
    while stack:
        bi, pcv = stack.pop()
        _, order, ncv, cvl = branches[bi]
        dia = diam_root + (diam_tip - diam_root) * (order / max_order if max_order else 0.0)
        for j in range(ncv):
            parent.append(pcv if j == 0 else len(parent) - 1)
            length.append(cvl)
            diam.append(dia)
        last = len(parent) - 1
        for ch in reversed(children[bi]):
            stack.append((ch, last))
    region = np.ones(len(parent), dtype=np.int32)
    region[0] = 0
    return Morphology(np.asarray(parent, np.int32), np.asarray(length), np.asarray(diam), region)


# --------------------------------------------------------------------------
# workloads
def single_neuron(dt: float = 0.025, seed: Optional[int] = None, w_syn: float = 1e-3,
                  sigma_pl: float = 0.0) -> Network:
    """Plain FP64 single ball-and-stick neuron with one calcium-plastic synapse at the
    dendrite midpoint, 10 Hz Poisson input and a 0.5 nA somatic step (sigma_pl:
    plasticity noise, Table 3's 2.8248 for the noisy variant)."""
    b = _Builder(dt, config_seed("single_neuron") if seed is None else seed, "single_neuron")
    hh = b.mech(HH, hh_params())
    pas = b.mech(PAS, pas_params(3e-5, -54.4))
    gb = b.mech(GB, gb_params(sigma_pl=sigma_pl))
    m = b.morph(ball_and_stick(20.0, 500.0, 1.0, 64))
    b.cells_add(1, m, hh, pas, istep=0.5)
    b.connect(SRC_POISSON, 0, 1 + 64 // 2, gb, w_syn, rate=10.0)
    return b.build()


def recurrent_stc(n_exc=1600, n_inh=400, p=0.1, dt=0.2, seed=None, w_bg=1e-3,
                  bg_rate=5.0, sigma_pl=0.0) -> Network:
    """Plain FP64 recurrent network: HH ball-and-stick cells with an 8-CV 200 um
    dendrite; Erdos-Renyi connectivity without self-loops; 3 ms delays; weights
    1 nS * U(0.9, 1.1); E->E synapses follow the tagging-and-capture rule; all
    other synapses are static; every cell receives 5 Hz Poisson background."""
    name = "recurrent_stc"
    b = _Builder(dt, config_seed(name) if seed is None else seed, name)
    rng = np.random.default_rng(b.seed)
    hh = b.mech(HH, hh_params())
    pas = b.mech(PAS, pas_params(3e-5, -54.4))
    exc = b.mech(EXPSYN, expsyn_params(5.0, 0.0))
    inh = b.mech(EXPSYN, expsyn_params(5.0, -80.0))
    stc = b.mech(STC, stc_params(sigma_pl=sigma_pl))
    m = b.morph(ball_and_stick(20.0, 200.0, 1.0, 8))
    n = n_exc + n_inh
    b.cells_add(n, m, hh, pas)
    adj = rng.random((n, n)) < p
    np.fill_diagonal(adj, False)
    src, dst = np.nonzero(adj)  # row-major: sorted by source
    w = 1e-3 * rng.uniform(0.9, 1.1, size=src.shape[0])
    e_src = src < n_exc
    mech = np.where(e_src, np.where(dst < n_exc, stc, exc), inh)
    cv = np.where(e_src, rng.integers(1, 9, size=src.shape[0]), 0)
    b.connect(src, dst, cv, mech, w, delay=3.0)
    b.connect(SRC_POISSON, np.arange(n), 0, exc, w_bg, rate=bg_rate)
    return b.build()


def stc_morpho_cell(large_cell: bool = False, large_dend: bool = False) -> Morphology:
    """Multi-compartment STC neuron of Table 6 (1 um compartments of one radius,
    6 or 12 um): the synthesis compartment (CV 0, the soma proper) between two
    halves of the somatic cylinder (l_soma / 2 each), the apical branch (12.5 or
    25 um) continuing one half and the basal branch (5 or 10 um) the other: 31
    or 48 CVs.  Only CV 0 is region 0 (the engine's HH is somatic)."""
    r = 12.0 if large_cell else 6.0
    half = int(round((24.0 if large_cell else 12.0) / 2))
    apical = 25.0 if large_dend else 12.5
    basal = 10.0 if large_dend else 5.0

    def pieces(total):
        n = int(np.floor(total))
        out = [1.0] * n
        if total - n > 1e-9:
            out.append(total - n)
        return out

    lengths = [1.0]
    parent = [-1]
    for branch in (apical, basal):
        prev = 0
        for ln in [1.0] * half + pieces(branch):
            parent.append(prev)
            lengths.append(ln)
            prev = len(lengths) - 1
    n = len(lengths)
    return Morphology(np.asarray(parent, np.int32), np.asarray(lengths),
                      np.full(n, 2.0 * r), np.r_[0, np.ones(n - 1)].astype(np.int32))


def recurrent_stc_morpho(n_exc=160, n_inh=40, p=0.1, dt=0.2, seed=None, d_p=1e-2,
                         large_cell=False, large_dend=False, w_ext=4e-3, ext_rate=40.0,
                         n_ext=4, w_rec=2e-3, w_inh=2e-3, sigma_pl=0.0,
                         tau_p=3600.0e3) -> Network:
    """Recurrent tagging-and-capture network of multi-compartment neurons
    (Sec. on memory consolidation in networks of morphological neurons): the
    excitatory cells have the morphology of stc_morpho_cell and a diffusing PRP
    (D_p, um2/ms; 1e-2 = 1e-11 m2/s); external Poisson input onto the apical
    tip, recurrent E->E (STC) synapses onto the basal tip, inhibition onto the
    soma; inhibitory cells are single-compartment.  HH soma, passive elsewhere;
    Erdos-Renyi connectivity without self-loops, 3 ms delays."""
    name = "recurrent_stc_morpho"
    b = _Builder(dt, config_seed(name) if seed is None else seed, name)
    rng = np.random.default_rng(b.seed)
    hh = b.mech(HH, hh_params())
    pas = b.mech(PAS, pas_params(3e-5, -54.4))
    exc = b.mech(EXPSYN, expsyn_params(5.0, 0.0))
    inh = b.mech(EXPSYN, expsyn_params(5.0, -80.0))
    stc = b.mech(STC, stc_params(sigma_pl=sigma_pl, d_p=d_p, tau_p=tau_p))
    mo = stc_morpho_cell(large_cell, large_dend)
    m_e = b.morph(mo)
    m_i = b.morph(soma_only(12.0))
    tips = [i for i in range(1, mo.n_cv) if i not in set(mo.parent.tolist())]
    apical_tip, basal_tip = tips[0], tips[1]
    b.cells_add(n_exc, m_e, hh, pas)
    b.cells_add(n_inh, m_i, hh, hh)
    n = n_exc + n_inh
    adj = rng.random((n, n)) < p
    np.fill_diagonal(adj, False)
    src, dst = np.nonzero(adj)
    e_src, e_dst = src < n_exc, dst < n_exc
    mech = np.where(e_src, np.where(e_dst, stc, exc), inh)
    cv = np.where(e_src & e_dst, basal_tip, 0)
    w = np.where(e_src, w_rec, w_inh) * rng.uniform(0.9, 1.1, size=src.shape[0])
    b.connect(src, dst, cv, mech, w, delay=3.0)
    ext_dst = np.repeat(np.arange(n), n_ext)
    ext_cv = np.where(ext_dst < n_exc, apical_tip, 0)
    b.connect(SRC_POISSON, ext_dst, ext_cv, exc, w_ext, rate=ext_rate)
    return b.build()


def heterosyn_dendrite(dt=0.025, seed=None, n_spikes=10, isi_ms=10.0, t0_ms=10.0,
                       active=(0, 2), **hca):
    """Heterosynaptic calcium plasticity on a dendritic branch (Sec. on
    heterosynaptic calcium-based plasticity, Table 4, Fig. 8): an 80 um
    dendrite of 1 um CVs (radius 1 um) spanning x = -40..40 um, CV 0 its root,
    with four spine heads (1 um long, radius 1 um) on the CVs holding x = -1,
    0, 1 and 3 um; an HCA synapse on each head.  The active spines (1 and 3 by
    default) receive a regular train (n_spikes every isi_ms from t0_ms) from a
    source cell whose spikes are replayed; the others get a silent Poisson
    source.  The membrane is passive: the calcium is decoupled from the cable.
    Returns the network and the replay list (gid, step)."""
    name = "heterosyn_dendrite"
    b = _Builder(dt, config_seed(name) if seed is None else seed, name)
    pas = b.mech(PAS, pas_params())
    m_hca = b.mech(HCA, hca_params(**hca))
    n_d = 80
    heads = [39, 40, 41, 43]                       # CVs holding x = -1, 0, 1, 3 um
    parent = np.r_[-1, np.arange(n_d - 1), heads].astype(np.int32)
    n = parent.shape[0]
    morph = Morphology(parent, np.ones(n), np.full(n, 2.0), np.r_[0, np.ones(n - 1)].astype(np.int32))
    m_d = b.morph(morph)
    m_s = b.morph(soma_only(10.0))
    b.cells_add(1, m_d, pas, pas)
    b.cells_add(1, m_s, pas, pas)                  # the replayed source, gid 1
    for k in range(4):
        if k in active:
            b.connect(1, 0, n_d + k, m_hca, 1.0, delay=dt)
        else:
            b.connect(SRC_POISSON, 0, n_d + k, m_hca, 1.0, rate=0.0)
    steps = np.array([int(round((t0_ms + j * isi_ms) / dt)) for j in range(n_spikes)], np.int64)
    return b.build(), (np.ones(n_spikes, np.int32), steps)


def morphology_sweep(n_nets=64, cells_per_net=500, p=0.1, dt=0.2, seed=None,
                     w_syn=1e-3, drive_hz=10.0) -> Network:
    """Many independent networks built like the single-neuron workload: per network a
    dendrite length L ~ U(100, 800) um with 4 + round(60 (L - 100) / 700) CVs and a
    diameter ~ U(0.5, 2) um; recurrent p, 3 ms delays, calcium-plastic synapses,
    10 Hz Poisson drive on the midpoint synapse and the 0.5 nA somatic step."""
    name = "morphology_sweep"
    b = _Builder(dt, config_seed(name) if seed is None else seed, name)
    rng = np.random.default_rng(b.seed)
    hh = b.mech(HH, hh_params())
    pas = b.mech(PAS, pas_params(3e-5, -54.4))
    gb = b.mech(GB, gb_params())
    for _ in range(n_nets):
        L = rng.uniform(100.0, 800.0)
        nd = 4 + int(round(60.0 * (L - 100.0) / 700.0))
        dia = rng.uniform(0.5, 2.0)
        m = b.morph(ball_and_stick(20.0, L, dia, nd))
        cells = b.cells_add(cells_per_net, m, hh, pas, istep=0.5)
        adj = rng.random((cells_per_net, cells_per_net)) < p
        np.fill_diagonal(adj, False)
        s, d = np.nonzero(adj)
        b.connect(cells[s], cells[d], rng.integers(1, nd + 1, size=s.shape[0]), gb, w_syn,
                  delay=3.0)
        b.connect(SRC_POISSON, cells, 1 + nd // 2, gb, w_syn, rate=drive_hz)
    return b.build()


def simple_branchy(rng: np.random.Generator, depth: int, soma_diam=20.0, cv_len=10.0,
                   diam=1.0, cvs_per_branch=9, p_fork=0.727) -> Morphology:
    """Random dendritic tree of the given depth on an HH soma (the busyring
    `simple-branchy` cell, Sec. "Runtime and memory benchmarking with
    large-scale networks").  Reading: two primary branches leave the soma; a
    branch of level l < depth forks into two with probability p_fork; every
    branch has cvs_per_branch CVs of cv_len um and diameter diam.  The defaults
    reproduce the mean compartment counts of Table 8 (45.0 per cell at depth 2,
    1633.5 at depth 10; one CV at depth 0).  Depth-first numbering."""
    parent, length, dia, region = [-1], [soma_diam], [soma_diam], [0]
    if depth <= 0:
        return Morphology(np.array(parent, np.int32), np.array(length), np.array(dia),
                          np.array(region, np.int32))
    stack = [(0, 1), (0, 1)]          # (parent CV, level); popped depth-first
    while stack:
        pcv, level = stack.pop()
        prev = pcv
        for _ in range(cvs_per_branch):
            parent.append(prev)
            length.append(cv_len)
            dia.append(diam)
            region.append(1)
            prev = len(parent) - 1
        if level < depth and rng.random() < p_fork:
            stack.append((prev, level + 1))
            stack.append((prev, level + 1))
    return Morphology(np.array(parent, np.int32), np.array(length), np.array(dia),
                      np.array(region, np.int32))


def busyring(n_cells=1024, depth=2, stdp=False, ring=4, s=1000, dt=0.025, delay_ms=5.0,
             w_ring=0.5, seed=None, n_shapes: Optional[int] = None) -> Network:
    """The busyring benchmark (Sec. "Runtime and memory benchmarking with large-scale
    networks", Table 7): rings of `ring` simple-branchy cells, each cell driving
    the next through an exponential synapse on the soma (tau 2 ms, E 0 mV,
    weight w_ring uS, delay 5 ms), so that a spike circulates at
    1 / (ring * delay); plus s random connections into every cell from random
    cells, weight 0, delay 5 ms, on uniform random CVs -- exponential synapses,
    or pair STDP (tau_pre = tau_post = 10 ms, A_pre 0.01, A_post -0.01,
    w_max 10, w0 0) with `stdp`.  The first cell of every ring is started by a
    2 nA, 1 ms somatic current step.  Each cell draws its own tree, or, with
    n_shapes, one of a pool of n_shapes trees (a faster generator for very large
    networks; the engine does not exploit shared shapes)."""
    name = f"busyring_d{depth}{'_stdp' if stdp else ''}"
    b = _Builder(dt, config_seed(name) if seed is None else seed, name)
    rng = np.random.default_rng(b.seed)
    hh = b.mech(HH, hh_params())
    pas = b.mech(PAS, pas_params(3e-5, -65.0))
    ring_syn = b.mech(EXPSYN, expsyn_params(2.0, 0.0))
    rand_syn = (b.mech(STDP, stdp_params(2.0, 0.0, 10.0, 10.0, 0.01, -0.01, 0.0, 10.0))
                if stdp else b.mech(EXPSYN, expsyn_params(2.0, 0.0)))
    n_trees = n_cells if n_shapes is None else min(n_shapes, n_cells)
    for _ in range(n_trees):
        b.morph(simple_branchy(rng, depth))
    tree_sizes = np.array([m.n_cv for m in b.morphs], np.int64)
    morph = np.arange(n_cells) if n_shapes is None else rng.integers(0, n_trees, n_cells)
    sizes = tree_sizes[morph]
    cells = np.arange(n_cells)
    first = cells % ring == 0
    b.cells_add(n_cells, morph, hh, pas, istep=np.where(first, 2.0, 0.0), ton=0.0,
                toff=np.where(first, 1.0, NEVER))
    nxt = (cells // ring) * ring + (cells % ring + 1) % ring
    b.connect(cells, nxt, 0, ring_syn, w_ring, delay=delay_ms)
    if s > 0:
        dst = np.repeat(cells, s)
        src = rng.integers(0, n_cells, size=dst.shape[0])
        cv = (rng.random(dst.shape[0]) * sizes[dst]).astype(np.int64)
        order = np.argsort(src, kind="stable")
        b.connect(src[order], dst[order], cv[order], rand_syn, 0.0, delay=delay_ms)
    return b.build()


def large_stdp(n_cells=100_000, fan_in=100, dt=0.025, seed=None, n_dend=(50, 500),
               w_syn=1e-3, w_drive=0.05, drive_hz=2.0, delay_ms=(1.0, 5.0),
               n_shapes: Optional[int] = None) -> Network:
    """Large network of HH-soma cells on random binary dendritic trees of 50-500
    dendritic CVs; fixed fan-in of `fan_in` uniform random presynaptic cells per
    cell with pair-STDP synapses on uniform random dendritic CVs and delays of
    1-5 ms; every cell also receives a 2 Hz Poisson drive on a static somatic
    synapse.  n_shapes, if given, draws that many tree shapes and assigns them
    to cells uniformly (a cheaper generator for very large networks)."""
    name = "large_stdp"
    b = _Builder(dt, config_seed(name) if seed is None else seed, name)
    rng = np.random.default_rng(b.seed)
    hh = b.mech(HH, hh_params())
    pas = b.mech(PAS, pas_params(3e-5, -54.4))
    stdp = b.mech(STDP, stdp_params())
    drive = b.mech(EXPSYN, expsyn_params(5.0, 0.0))
    n_trees = n_cells if n_shapes is None else n_shapes
    tree_sizes = rng.integers(n_dend[0], n_dend[1] + 1, size=n_trees)
    for t in range(n_trees):
        b.morph(random_binary_tree(rng, int(tree_sizes[t])))
    morph_ids = np.arange(n_cells) if n_shapes is None else rng.integers(0, n_trees, n_cells)
    sizes = tree_sizes[morph_ids]
    cells = b.cells_add(n_cells, morph_ids, hh, pas)
    src = rng.integers(0, n_cells - 1, size=(n_cells, fan_in))
    src = (src + (src >= cells[:, None])).reshape(-1)   # no self-connections
    dst = np.repeat(cells, fan_in)
    cv = 1 + (rng.random(dst.shape[0]) * sizes[dst]).astype(np.int64)
    steps = rng.integers(int(round(delay_ms[0] / dt)), int(round(delay_ms[1] / dt)) + 1,
                         size=dst.shape[0])
    order = np.argsort(src, kind="stable")
    b.connect(src[order], dst[order], cv[order], stdp, w_syn, delay=steps[order] * dt)
    b.connect(SRC_POISSON, cells, 0, drive, w_drive, rate=drive_hz)
    return b.build()


def serving_job(n_cells: int, long_dendrite: bool, dend_len_um: float, dend_diam_um: float,
                seed: int, dt: float = 0.2, fan_in: int = 50, w_syn: float = 1e-3,
                w_bg: float = 3e-3, bg_rate: float = 20.0) -> Network:
    """One serving job: n_cells HH ball-and-stick cells (a 64-CV dendrite like the
    single-neuron workload, or an 8-CV one like the recurrent network) with the
    job's dendritic length and diameter (a parameter sweep), random recurrent
    connectivity of fan-in min(fan_in, n_cells - 1) with 3 ms delays and pair-STDP
    synapses, and Poisson background on a somatic synapse."""
    b = _Builder(dt, seed, "serving_job")
    rng = np.random.default_rng(seed)
    hh = b.mech(HH, hh_params())
    pas = b.mech(PAS, pas_params(3e-5, -54.4))
    bg = b.mech(EXPSYN, expsyn_params(5.0, 0.0))
    stdp = b.mech(STDP, stdp_params())
    nd = 64 if long_dendrite else 8
    m = b.morph(ball_and_stick(20.0, dend_len_um, dend_diam_um, nd))
    cells = b.cells_add(n_cells, m, hh, pas)
    k = min(fan_in, n_cells - 1)
    if k > 0:
        src = rng.integers(0, n_cells - 1, size=(n_cells, k))
        src = (src + (src >= cells[:, None])).reshape(-1)
        dst = np.repeat(cells, k)
        b.connect(src, dst, rng.integers(1, nd + 1, size=dst.shape[0]), stdp, w_syn, delay=3.0)
    b.connect(SRC_POISSON, cells, 0, bg, w_bg, rate=bg_rate)
    return b.build()


def serving_trace(n_jobs: int = 2000, rate_hz: float = 20.0, seed: Optional[int] = None,
                  sizes=(1, 20000), durations_s=(0.1, 10.0), dt: float = 0.2):
    """Poisson arrivals of serving jobs: sizes log-uniform in `sizes` cells, durations
    log-uniform in `durations_s` simulated seconds, 64-CV and 8-CV morphologies 50/50,
    dendrite length U(100, 800) um and diameter U(0.5, 2) um per job."""
    rng = np.random.default_rng(config_seed("serving") if seed is None else seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n_jobs))
    lo, hi = np.log(sizes[0]), np.log(sizes[1])
    n = np.floor(np.exp(rng.uniform(lo, np.log(sizes[1] + 1), size=n_jobs))).astype(int)
    n = np.clip(n, sizes[0], sizes[1])
    dur = np.exp(rng.uniform(np.log(durations_s[0]), np.log(durations_s[1]), size=n_jobs))
    long_d = rng.random(n_jobs) < 0.5
    L = rng.uniform(100.0, 800.0, size=n_jobs)
    d = rng.uniform(0.5, 2.0, size=n_jobs)
    seeds = rng.integers(0, 2**62, size=n_jobs)
    return [dict(job_id=i, arrival_s=float(t[i]), n_cells=int(n[i]), long_dendrite=bool(long_d[i]),
                 dend_len_um=float(L[i]), dend_diam_um=float(d[i]),
                 duration_ms=float(round(dur[i] * 1000.0 / dt) * dt), seed=int(seeds[i]), dt=dt)
            for i in range(n_jobs)]
