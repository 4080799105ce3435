"""ctypes loader for the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py.  The product package never imports this module.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .build_oracle import LIB, build

_lib = None

SYN_G, SYN_C, SYN_W, SYN_H, SYN_Z, SYN_APRE, SYN_APOST, SYN_WEIGHT_TOTAL = range(8)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        P = C.c_void_p
        L.orc_build.restype = C.c_int
        L.orc_build.argtypes = ([C.c_int32] + [P] * 10 + [C.c_int32] + [P] * 6 + [C.c_int32]
                                + [P] * 3 + [C.c_int64] + [C.c_int64] + [P] * 8
                                + [C.c_double, C.c_uint64, C.c_int32, P, P, P])
        L.orc_run.argtypes = [P, C.c_int64]
        L.orc_set_replay.argtypes = [P, C.c_int64, P, P]
        L.orc_inject_spikes.argtypes = [P, C.c_int64, P, P]
        for fn in ("orc_n_spikes", "orc_n_cv", "orc_n_probe_samples", "orc_step_count"):
            getattr(L, fn).restype = C.c_int64
            getattr(L, fn).argtypes = [P]
        L.orc_get_spikes.argtypes = [P, P, P, P]
        L.orc_get_v.argtypes = [P, P]
        L.orc_get_probes.argtypes = [P, P]
        L.orc_get_syn.argtypes = [P, C.c_int32, P]
        L.orc_get_cell_p.argtypes = [P, P]
        L.orc_get_prp.argtypes = [P, P]
        L.orc_get_ca.argtypes = [P, P]
        L.orc_set_ca.argtypes = [P, P]
        L.orc_set_prp.argtypes = [P, P]
        L.orc_has_diffusion.restype = C.c_int32
        L.orc_has_diffusion.argtypes = [P, C.c_int32]
        L.orc_get_gates.argtypes = [P, P]
        L.orc_get_cv_geometry.argtypes = [P, P, P, P]
        L.orc_fast_forward.argtypes = [P, C.c_int64, C.c_int64]
        L.orc_set_syn.argtypes = [P, C.c_int32, P]
        for fn in ("orc_set_v", "orc_set_cell_p", "orc_set_gates"):
            getattr(L, fn).argtypes = [P, P]
        L.orc_free.argtypes = [P]
        L.orc_last_error.restype = C.c_char_p
        L.orc_exp.restype = C.c_double
        L.orc_exp.argtypes = [C.c_double]
        L.orc_hh_rates.argtypes = [C.c_double] + [P] * 6
        L.orc_hines_solve.argtypes = [C.c_int32, P, P, P, P, P]
        L.orc_threefry4x64_12.argtypes = [P, P, P]
        L.orc_poisson_u32.restype = C.c_uint32
        L.orc_poisson_u32.argtypes = [C.c_uint64, C.c_uint64, C.c_int64]
        L.orc_log.restype = C.c_double
        L.orc_log.argtypes = [C.c_double]
        L.orc_cis2pi.restype = C.c_double
        L.orc_cis2pi.argtypes = [C.c_double, C.c_int]
        L.orc_normal.restype = C.c_double
        L.orc_normal.argtypes = [C.c_uint64, C.c_uint64, C.c_int64]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One oracle model built from a workloads.Network."""

    def __init__(self, net, probes=()):
        L = lib()
        keep = []

        def arr(x, dt):
            a = np.ascontiguousarray(np.asarray(x), dtype=dt)
            keep.append(a)
            return _p(a)

        ncv, moff, par, ln, dm, reg = net.packed_morphs()
        mk, mo, mp = net.packed_mechs()
        pg = np.array([p[0] for p in probes], dtype=np.int32)
        pc = np.array([p[1] for p in probes], dtype=np.int32)
        h = C.c_void_p()
        rc = L.orc_build(
            net.n_cells, arr(net.cell_morph, np.int32), arr(net.cell_soma_mech, np.int32),
            arr(net.cell_dend_mech, np.int32), arr(net.cell_cm, np.float64),
            arr(net.cell_ra, np.float64), arr(net.cell_istep, np.float64),
            arr(net.cell_ton, np.float64), arr(net.cell_toff, np.float64),
            arr(net.cell_vinit, np.float64), arr(net.cell_thresh, np.float64),
            len(net.morphs), arr(ncv, np.int32), arr(moff, np.int32), arr(par, np.int32),
            arr(ln, np.float64), arr(dm, np.float64), arr(reg, np.int32),
            len(mk), arr(mk, np.int32), arr(mo, np.int32), arr(mp, np.float64), len(mp),
            net.n_conn, arr(net.conn_src, np.int32), arr(net.conn_dst, np.int32),
            arr(net.conn_cv, np.int32), arr(net.conn_mech, np.int32),
            arr(net.conn_weight, np.float64), arr(net.conn_delay, np.float64),
            arr(net.conn_rate, np.float64), arr(net.conn_pid, np.int64), float(net.dt), int(net.seed) & (2**64 - 1),
            len(pg), arr(pg, np.int32), arr(pc, np.int32), C.byref(h))
        if rc != 0:
            raise ValueError("oracle build failed: " + L.orc_last_error().decode())
        self._h = h
        self.n_cells = net.n_cells
        self.n_conn = net.n_conn
        self.n_probe = len(pg)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_free(h)
            self._h = None

    def set_replay(self, gid, step):
        gid = np.ascontiguousarray(gid, dtype=np.int32)
        step = np.ascontiguousarray(step, dtype=np.int64)
        if lib().orc_set_replay(self._h, len(gid), _p(gid), _p(step)) != 0:
            raise ValueError(lib().orc_last_error().decode())

    def inject_spikes(self, gid, step):
        """Spikes of cells simulated elsewhere (past steps; their events still due)."""
        gid = np.ascontiguousarray(gid, dtype=np.int32)
        step = np.ascontiguousarray(step, dtype=np.int64)
        if lib().orc_inject_spikes(self._h, len(gid), _p(gid), _p(step)) != 0:
            raise ValueError(lib().orc_last_error().decode())

    def run(self, n_steps: int):
        lib().orc_run(self._h, int(n_steps))

    @property
    def step(self) -> int:
        return lib().orc_step_count(self._h)

    def spikes(self):
        n = lib().orc_n_spikes(self._h)
        gid = np.zeros(n, np.int32)
        step = np.zeros(n, np.int64)
        t = np.zeros(n, np.float64)
        lib().orc_get_spikes(self._h, _p(gid), _p(step), _p(t))
        return gid, step, t

    def v(self):
        out = np.zeros(lib().orc_n_cv(self._h))
        lib().orc_get_v(self._h, _p(out))
        return out

    def probes(self):
        ns = lib().orc_n_probe_samples(self._h)
        out = np.zeros(ns * self.n_probe)
        lib().orc_get_probes(self._h, _p(out))
        return out.reshape(ns, self.n_probe)

    def step_count(self) -> int:
        return int(lib().orc_step_count(self._h))

    def fast_forward(self, steps: int, n_long: int):
        """steps of simulated time without spiking and calcium dynamics, the slow
        plasticity variables in n_long long forward-Euler steps."""
        if lib().orc_fast_forward(self._h, steps, n_long) != 0:
            raise ValueError("fast_forward: bad arguments or replay mode")

    def set_syn(self, field: int, values):
        a = np.ascontiguousarray(values, np.float64)
        assert a.shape == (self.n_conn,)
        lib().orc_set_syn(self._h, field, _p(a))

    def set_v(self, values):
        a = np.ascontiguousarray(values, np.float64)
        lib().orc_set_v(self._h, _p(a))

    def set_cell_p(self, values):
        a = np.ascontiguousarray(values, np.float64)
        assert a.shape == (self.n_cells,)
        lib().orc_set_cell_p(self._h, _p(a))

    def set_gates(self, values):
        a = np.ascontiguousarray(values, np.float64).reshape(-1)
        assert a.shape == (3 * self.n_cells,)
        lib().orc_set_gates(self._h, _p(a))

    def syn(self, field: int):
        out = np.zeros(self.n_conn)
        lib().orc_get_syn(self._h, int(field), _p(out))
        return out

    def cell_p(self):
        out = np.zeros(self.n_cells)
        lib().orc_get_cell_p(self._h, _p(out))
        return out

    def prp(self):
        """PRP concentration per CV (cell-major) of the cells whose PRP diffuses;
        0 on every other CV."""
        out = np.zeros(lib().orc_n_cv(self._h))
        lib().orc_get_prp(self._h, _p(out))
        return out

    def set_prp(self, values):
        a = np.ascontiguousarray(values, np.float64)
        assert a.shape == (lib().orc_n_cv(self._h),)
        lib().orc_set_prp(self._h, _p(a))

    def ca(self):
        """Heterosynaptic calcium per CV (cell-major) of cells with HCA synapses
        [umol/l]; 0 on every other CV."""
        out = np.zeros(lib().orc_n_cv(self._h))
        lib().orc_get_ca(self._h, _p(out))
        return out

    def set_ca(self, values):
        a = np.ascontiguousarray(values, np.float64)
        assert a.shape == (lib().orc_n_cv(self._h),)
        lib().orc_set_ca(self._h, _p(a))

    def has_diffusion(self, cell: int) -> bool:
        return bool(lib().orc_has_diffusion(self._h, int(cell)))

    def gates(self):
        out = np.zeros(3 * self.n_cells)
        lib().orc_get_gates(self._h, _p(out))
        return out.reshape(self.n_cells, 3)

    def geometry(self):
        n = lib().orc_n_cv(self._h)
        cap, gp, a = np.zeros(n), np.zeros(n), np.zeros(n)
        lib().orc_get_cv_geometry(self._h, _p(cap), _p(gp), _p(a))
        return cap, gp, a


def exp(x: float) -> float:
    return lib().orc_exp(float(x))


def hh_rates(v: float):
    vals = [C.c_double() for _ in range(6)]
    lib().orc_hh_rates(float(v), *[C.byref(x) for x in vals])
    return tuple(x.value for x in vals)


def hines_solve(parent, d, a, b):
    n = len(d)
    parent = np.ascontiguousarray(parent, np.int32)
    d = np.ascontiguousarray(d, np.float64)
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros(n)
    rc = lib().orc_hines_solve(n, _p(parent), _p(d), _p(a), _p(b), _p(x))
    assert rc == 0
    return x


def threefry(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint64)
    k = np.ascontiguousarray(key, np.uint64)
    o = np.zeros(4, np.uint64)
    lib().orc_threefry4x64_12(_p(c), _p(k), _p(o))
    return o


def poisson_u32(seed: int, stream: int, step: int) -> int:
    return lib().orc_poisson_u32(seed & (2**64 - 1), stream, step)


def log(x: float) -> float:
    return lib().orc_log(float(x))


def cis2pi(v: float, which: int) -> float:
    """cos(2 pi v) (which = 0) or sin(2 pi v) (which = 1), the model's own."""
    return lib().orc_cis2pi(float(v), int(which))


def normal(seed: int, noise_id: int, step: int) -> float:
    return lib().orc_normal(seed & (2**64 - 1), noise_id, step)
