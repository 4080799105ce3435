"""Thin ctypes binding of libplasticarbor.so (include/plastic_arbor.h).

Argument marshalling only: every step of the simulation runs in the library's
CUDA kernels.  There is no CPU fallback: if the shared library is missing or
no CUDA device is visible, building a model raises.
"""
from __future__ import annotations

import ctypes as C
import os
from concurrent.futures import ThreadPoolExecutor
from typing import Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PA_LIBRARY selects another build of the library (the bounds-checked one in
# its tests); by default the in-tree libplasticarbor.so
LIB_PATH = os.environ.get("PA_LIBRARY") or os.path.join(HERE, "libplasticarbor.so")

PA_FP64, PA_MIXED, PA_FP32 = 0, 1, 2
PA_SRC_POISSON = -1
FIELD_G, FIELD_C, FIELD_W, FIELD_H, FIELD_Z, FIELD_APRE, FIELD_APOST = range(7)
FIELD_V, FIELD_PRP, FIELD_GATES, FIELD_PRP_CV, FIELD_CA_CV = 16, 17, 18, 19, 20
ERRORS = {-1: "PA_ERR_ARG", -2: "PA_ERR_OOM", -3: "PA_ERR_CUDA", -4: "PA_ERR_TIMEOUT",
          -5: "PA_ERR_CAPACITY", -6: "PA_ERR_STATE"}

EXPORTED = ("pa_build_model", "pa_advance", "pa_advance_noalloc", "pa_sync", "pa_set_wait_limit",
            "pa_read_probes", "pa_read_spikes",
            "pa_read_weights", "pa_read_state", "pa_set_replay", "pa_model_info",
            "pa_get_kernel_stats", "pa_reset_kernel_stats", "pa_get_tuning", "pa_free_model",
            "pa_check_arith", "pa_measure_fp64", "pa_write_state", "pa_fast_forward",
            "pa_inject_spikes", "pa_batch_create", "pa_batch_add", "pa_batch_remove",
            "pa_batch_advance", "pa_batch_info", "pa_batch_free",
            "pa_last_error")


class PaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Morph(C.Structure):
    _fields_ = [("n_cv", C.c_int32), ("parent", C.c_void_p), ("length_um", C.c_void_p),
                ("diam_um", C.c_void_p), ("region", C.c_void_p)]


# the same layout as Morph, for building the whole table with numpy
MORPH_DTYPE = np.dtype({"names": [f[0] for f in Morph._fields_],
                        "formats": ["<i4", "<u8", "<u8", "<u8", "<u8"],
                        "offsets": [getattr(Morph, f[0]).offset for f in Morph._fields_],
                        "itemsize": C.sizeof(Morph)})


def _morph_table(morphs, keep):
    """pa_morphology descriptors of every morphology, pointing into four
    concatenated arrays (appended to keep, which must outlive the call)."""
    tab = np.zeros(max(len(morphs), 1), MORPH_DTYPE)
    if not morphs:
        return tab
    k = len(morphs)
    off = np.zeros(k, np.int64)
    for f, src, dt in (("parent", "parent", np.int32), ("length_um", "length", np.float64),
                       ("diam_um", "diam", np.float64), ("region", "region", np.int32)):
        parts = [getattr(m, src) for m in morphs]
        n = np.fromiter(map(len, parts), np.int64, k)
        if f == "parent":
            tab["n_cv"] = n
            np.cumsum(n[:-1], out=off[1:])
        elif not np.array_equal(n, tab["n_cv"]):
            raise ValueError(f"morphology {src} arrays must have n_cv entries")
        a = np.concatenate(parts + [np.zeros(1, dt)], dtype=dt)
        keep.append(a)
        tab[f] = a.ctypes.data + a.itemsize * off
    return tab


def _pack(dtype, n: int, columns: dict) -> np.ndarray:
    """A structured array of n records from per-field columns.  Large tables are
    filled in row chunks on a few threads (numpy copies release the GIL)."""
    out = np.empty(n, dtype)
    chunk = 1 << 20
    if n <= 2 * chunk:
        for f, col in columns.items():
            out[f] = col
        return out

    def fill(i):
        sl = slice(i, min(i + chunk, n))
        for f, col in columns.items():
            out[f][sl] = np.asarray(col)[sl]

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        list(ex.map(fill, range(0, n, chunk)))
    return out


class Mech(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_params", C.c_int32), ("params", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("dt", C.c_double), ("seed", C.c_uint64), ("precision", C.c_int32),
                ("device", C.c_int32), ("stream", C.c_void_p), ("n_probe", C.c_int32),
                ("probe_gid", C.c_void_p), ("probe_cv", C.c_void_p),
                ("probe_capacity", C.c_int64), ("spike_capacity", C.c_int64),
                ("max_epoch_steps", C.c_int32), ("flags", C.c_int32)]


class KernelStats(C.Structure):
    _fields_ = [("epoch_launches", C.c_int64), ("kernel_launches", C.c_int64),
                ("epoch_kernel_ms", C.c_double), ("event_kernels_ms", C.c_double),
                ("graph_launches", C.c_int64)]


FLAG_TIME_KERNELS = 1
FLAG_AUTOTUNE = 2
FLAG_NO_GRAPHS = 8
FLAG_NARROW_ONLY = 16
FLAG_WIDE_ALL = 32


def FLAG_BUILD_THREADS(n: int) -> int:
    """at most n host threads for the model's build (0: automatic)"""
    return (int(n) & 0x3F) << 12
N_SHAPES = 6


def flag_shape(s: int) -> int:
    """pa_options.flags value forcing epoch-kernel shape s."""
    return ((s + 1) & 0xF) << 8


class Info(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_cv", C.c_int64), ("n_conn", C.c_int64),
                ("n_groups", C.c_int64), ("n_padded_cv", C.c_int64), ("step", C.c_int64),
                ("epoch_steps", C.c_int32), ("precision", C.c_int32), ("tree", C.c_int32),
                ("n_streams", C.c_int32), ("shape", C.c_int32), ("n_wide", C.c_int32),
                ("device_bytes", C.c_int64), ("n_static_cv", C.c_int64)]


CELL_DTYPE = np.dtype([("morph", "<i4"), ("soma_mech", "<i4"), ("dend_mech", "<i4"),
                       ("reserved", "<i4"), ("cm", "<f8"), ("ra", "<f8"), ("i_step", "<f8"),
                       ("t_on", "<f8"), ("t_off", "<f8"), ("v_init", "<f8"),
                       ("threshold", "<f8")])
CONN_DTYPE = np.dtype([("src_gid", "<i4"), ("dst_gid", "<i4"), ("dst_cv", "<i4"),
                       ("mech", "<i4"), ("weight", "<f8"), ("delay_ms", "<f8"),
                       ("rate_hz", "<f8"), ("poisson_id", "<i8")])

_lib = None


def lib():
    """Loads the engine library (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2411_16445_b300/build_lib.py")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.pa_build_model.argtypes = [P, C.c_int64, P, C.c_int64, P, C.c_int64, P, C.c_int64,
                                     P, C.POINTER(C.c_void_p)]
        L.pa_advance.argtypes = [P, C.c_double, C.c_double]
        L.pa_advance_noalloc.argtypes = [P, C.c_double, C.c_double]
        L.pa_sync.argtypes = [P]
        L.pa_set_wait_limit.argtypes = [P, C.c_uint32]
        L.pa_read_probes.argtypes = [P, P, C.c_int64, C.POINTER(C.c_int64)]
        L.pa_read_spikes.argtypes = [P, P, P, P, C.c_int64, C.POINTER(C.c_int64)]
        L.pa_read_weights.argtypes = [P, P, C.c_int64, C.POINTER(C.c_int64)]
        L.pa_read_state.argtypes = [P, C.c_int32, P, C.c_int64, C.POINTER(C.c_int64)]
        L.pa_set_replay.argtypes = [P, C.c_int64, P, P]
        L.pa_inject_spikes.argtypes = [P, C.c_int64, P, P]
        L.pa_batch_create.argtypes = [C.c_int32, P, C.POINTER(C.c_void_p)]
        L.pa_batch_add.argtypes = [P, P]
        L.pa_batch_remove.argtypes = [P, P]
        L.pa_batch_advance.argtypes = [P, C.c_int64]
        L.pa_batch_info.argtypes = [P, P]
        L.pa_batch_free.argtypes = [P]
        L.pa_batch_free.restype = None
        L.pa_model_info.argtypes = [P, C.POINTER(Info)]
        L.pa_get_kernel_stats.argtypes = [P, C.POINTER(KernelStats)]
        L.pa_reset_kernel_stats.argtypes = [P]
        L.pa_get_tuning.argtypes = [P, C.POINTER(C.c_int32), P, C.c_int32]
        L.pa_check_arith.argtypes = [C.c_int32, C.c_uint64, C.c_int64, P]
        L.pa_measure_fp64.argtypes = [C.c_int32, P]
        L.pa_write_state.argtypes = [P, C.c_int32, P, C.c_int64]
        L.pa_fast_forward.argtypes = [P, C.c_double, C.c_int64]
        L.pa_free_model.argtypes = [P]
        L.pa_free_model.restype = None
        L.pa_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise PaError(rc, lib().pa_last_error().decode())


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data) if a.size else C.c_void_p(0)


def check_arith(device: int = 0, seed: int = 1, n_random: int = 1 << 30) -> dict:
    """pa_check_arith: the integer FP64 reciprocal and float widening against the
    GPU's IEEE operations; returns the mismatch counts."""
    out = np.zeros(4, np.int64)
    _check(lib().pa_check_arith(device, seed, n_random, _ptr(out)))
    return {"rcp_mismatch": int(out[0]), "widen_mismatch": int(out[1]),
            "checked": int(out[2]), "first_bad_rcp_bits": int(out[3])}


def measure_fp64(device: int = 0) -> dict:
    """pa_measure_fp64: the GPU's FP64 FMA throughput (FMA/s) and the best run's ms."""
    out = np.zeros(2)
    _check(lib().pa_measure_fp64(device, _ptr(out)))
    return {"fma_per_s": float(out[0]), "ms": float(out[1])}


def current_stream_handle(device: int = 0):
    """cudaStream_t of torch's current stream on `device` (0 = legacy default)."""
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    except Exception:
        pass
    return C.c_void_p(0)


class Model:
    """A network resident on the GPU.  Mirrors pa_build_model .. pa_free_model."""

    def __init__(self, net, precision: int = PA_FP64, probes: Sequence[Tuple[int, int]] = (),
                 device: int = 0, stream=None, probe_capacity: int = 0,
                 spike_capacity: int = 0, max_epoch_steps: int = 0, flags: int = 0):
        L = lib()
        keep = []
        cells = np.zeros(net.n_cells, CELL_DTYPE)
        cells["morph"], cells["soma_mech"], cells["dend_mech"] = (
            net.cell_morph, net.cell_soma_mech, net.cell_dend_mech)
        for f, src in (("cm", net.cell_cm), ("ra", net.cell_ra), ("i_step", net.cell_istep),
                       ("t_on", net.cell_ton), ("t_off", net.cell_toff),
                       ("v_init", net.cell_vinit), ("threshold", net.cell_thresh)):
            cells[f] = src
        morphs = _morph_table(net.morphs, keep)
        mechs = (Mech * max(len(net.mech_params), 1))()
        for i, (k, p) in enumerate(zip(net.mech_kind, net.mech_params)):
            pa = np.ascontiguousarray(p, np.float64)
            keep.append(pa)
            mechs[i] = Mech(int(k), len(pa), pa.ctypes.data)
        conns = _pack(CONN_DTYPE, net.n_conn, {
            "src_gid": net.conn_src, "dst_gid": net.conn_dst, "dst_cv": net.conn_cv,
            "mech": net.conn_mech, "weight": net.conn_weight, "delay_ms": net.conn_delay,
            "rate_hz": net.conn_rate, "poisson_id": net.conn_pid})
        pg = np.ascontiguousarray([p[0] for p in probes], np.int32)
        pc = np.ascontiguousarray([p[1] for p in probes], np.int32)
        if stream is None:
            stream = current_stream_handle(device)
        opt = Options(dt=float(net.dt), seed=int(net.seed) & (2**64 - 1), precision=precision,
                      device=device, stream=stream, n_probe=len(pg),
                      probe_gid=pg.ctypes.data if len(pg) else None,
                      probe_cv=pc.ctypes.data if len(pc) else None,
                      probe_capacity=probe_capacity, spike_capacity=spike_capacity,
                      max_epoch_steps=max_epoch_steps, flags=flags)
        h = C.c_void_p()
        _check(L.pa_build_model(_ptr(cells), net.n_cells, _ptr(morphs),
                                len(net.morphs), C.cast(mechs, C.c_void_p),
                                len(net.mech_params), _ptr(conns), net.n_conn,
                                C.byref(opt), C.byref(h)))
        self._h = h
        self.dt = float(net.dt)
        self.n_conn = net.n_conn
        self.n_cells = net.n_cells

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.pa_free_model(self._h)
            self._h = None

    __del__ = close

    def info(self) -> Info:
        inf = Info()
        _check(lib().pa_model_info(self._h, C.byref(inf)))
        return inf

    @property
    def step(self) -> int:
        return int(self.info().step)

    def advance(self, t_end_ms: float):
        _check(lib().pa_advance(self._h, float(t_end_ms), self.dt))

    def advance_noalloc(self, t_end_ms: float):
        """pa_advance_noalloc: same as advance(), allocating nothing during the call."""
        _check(lib().pa_advance_noalloc(self._h, float(t_end_ms), self.dt))

    def advance_steps(self, n: int):
        self.advance((self.step + int(n)) * self.dt)

    def sync(self):
        _check(lib().pa_sync(self._h))

    def set_wait_limit(self, polls: int):
        """pa_set_wait_limit: polls of the bounded row-staging waits (0: default)."""
        _check(lib().pa_set_wait_limit(self._h, int(polls)))

    def read_probes(self, n_probe: int) -> np.ndarray:
        n = C.c_int64()
        _check(lib().pa_read_probes(self._h, None, 0, C.byref(n)))
        out = np.zeros(n.value)
        if n.value:
            _check(lib().pa_read_probes(self._h, _ptr(out), n.value, C.byref(n)))
        return out.reshape(-1, n_probe) if n_probe else out

    def read_spikes(self):
        n = C.c_int64()
        _check(lib().pa_read_spikes(self._h, None, None, None, 0, C.byref(n)))
        gid = np.zeros(n.value, np.int32)
        step = np.zeros(n.value, np.int64)
        t = np.zeros(n.value)
        if n.value:
            _check(lib().pa_read_spikes(self._h, _ptr(gid), _ptr(step), _ptr(t), n.value,
                                        C.byref(n)))
        return gid, step, t

    def read_weights(self) -> np.ndarray:
        out = np.zeros(self.n_conn)
        n = C.c_int64()
        _check(lib().pa_read_weights(self._h, _ptr(out), len(out), C.byref(n)))
        return out

    def read_state(self, field: int) -> np.ndarray:
        n = C.c_int64()
        _check(lib().pa_read_state(self._h, int(field), None, 0, C.byref(n)))
        out = np.zeros(n.value)
        _check(lib().pa_read_state(self._h, int(field), _ptr(out), n.value, C.byref(n)))
        return out

    def write_state(self, field: int, values) -> None:
        """pa_write_state: the inverse of read_state (same layout)."""
        a = np.ascontiguousarray(values, np.float64).reshape(-1)
        _check(lib().pa_write_state(self._h, int(field), _ptr(a), a.size))

    def fast_forward(self, duration_ms: float, n_long: int) -> None:
        """pa_fast_forward: duration_ms without spiking and calcium dynamics, the
        slow plasticity variables in n_long long steps."""
        _check(lib().pa_fast_forward(self._h, float(duration_ms), int(n_long)))

    def kernel_stats(self) -> KernelStats:
        ks = KernelStats()
        _check(lib().pa_get_kernel_stats(self._h, C.byref(ks)))
        return ks

    def tuning(self):
        """(shape in use, trial time in ms of each shape; zeros unless autotuned)"""
        s = C.c_int32()
        ms = np.zeros(N_SHAPES)
        _check(lib().pa_get_tuning(self._h, C.byref(s), _ptr(ms), N_SHAPES))
        return int(s.value), ms

    def reset_kernel_stats(self):
        _check(lib().pa_reset_kernel_stats(self._h))

    def inject_spikes(self, gid, step):
        """pa_inject_spikes: spikes of cells simulated elsewhere, in the last epoch."""
        gid = np.ascontiguousarray(gid, np.int32)
        step = np.ascontiguousarray(step, np.int64)
        _check(lib().pa_inject_spikes(self._h, len(gid), _ptr(gid), _ptr(step)))

    def set_replay(self, gid, step):
        gid = np.ascontiguousarray(gid, np.int32)
        step = np.ascontiguousarray(step, np.int64)
        _check(lib().pa_set_replay(self._h, len(gid), _ptr(gid), _ptr(step)))


class Batch:
    """Resident models advanced together, one grouped time-step launch per epoch
    (pa_batch_*).  Members run on the batch's stream."""

    def __init__(self, device: int = 0, stream=None):
        L = lib()
        if stream is None:
            stream = current_stream_handle(device)
        h = C.c_void_p()
        _check(L.pa_batch_create(device, stream, C.byref(h)))
        self._h = h
        self.members = []

    def add(self, model: "Model"):
        _check(lib().pa_batch_add(self._h, model._h))
        self.members.append(model)

    def remove(self, model: "Model"):
        _check(lib().pa_batch_remove(self._h, model._h))
        self.members.remove(model)

    def advance_epochs(self, n: int):
        _check(lib().pa_batch_advance(self._h, int(n)))

    def info(self):
        out = np.zeros(4, np.int64)
        _check(lib().pa_batch_info(self._h, _ptr(out)))
        return {"members": int(out[0]), "blocks": int(out[1]), "graph_launches": int(out[2]),
                "captures": int(out[3])}

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.pa_batch_free(self._h)
            self._h = None

    __del__ = close
