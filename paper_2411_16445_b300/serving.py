"""Continuous-batching simulation server on one GPU.

Jobs (one network each) arrive over time.  The server admits a job as soon as
the HBM budget allows, builds it on a background thread (pa_build_model), and
keeps its state resident.  It advances every resident job in fixed quanta of
simulated time, each job on its own CUDA stream, so the kernels of all resident
jobs overlap on the device.  A finished job's spikes and weights are read back
and its memory freed, which makes room for waiting jobs.  Latency is measured
from a job's arrival to the moment its results are on the host.

Quanta are whole 8-epoch CUDA-graph launches, more of them for a small job
(about `quantum_cu` compartment-updates per quantum; measured on the serving
trace, one launch per quantum for all but the smallest jobs keeps the large
jobs' kernels interleaved best).  Many jobs means
many streams: set CUDA_DEVICE_MAX_CONNECTIONS (32) before CUDA is initialised
so that their launches do not share a few hardware queues.

Jobs never share device state, so a job's results are the same whether it runs
alone or among others; tests/test_serving.py checks this.
"""
from __future__ import annotations

import dataclasses
import time
import zlib
from concurrent.futures import ThreadPoolExecutor
from typing import Dict, List, Optional

import numpy as np

from . import engine as E
from . import workloads as W


@dataclasses.dataclass
class JobResult:
    job_id: int
    arrival_s: float
    start_s: float
    done_s: float
    n_cv: int
    steps: int
    spikes: int
    spike_digest: int
    weights: np.ndarray

    @property
    def latency_s(self) -> float:
        return self.done_s - self.arrival_s


def estimate_bytes(net) -> int:
    """Upper bound of a model's device bytes: per padded CV the FP64 row arrays and
    scratch, per synapse its state and event words (ring of epochs)."""
    n_cv = net.n_cv + 32 * max(net.cell_ncv().max(initial=1), 1)
    rec = net.conn_src >= 0
    max_d = float(net.conn_delay[rec].max()) if rec.any() else 0.0
    min_d = float(net.conn_delay[rec].min()) if rec.any() else 64 * net.dt
    e = max(1, min(64, int(round(min_d / net.dt))))
    slots = int((max_d / net.dt + 100) / e) + 3
    return int(1.25 * (n_cv * 96 + net.n_conn * (72 + 16 * slots) + net.n_cells * 256) + (8 << 20))


def estimate_spec_bytes(spec, fan_in: int = 50) -> int:
    """estimate_bytes for a serving job, from its description alone."""
    nd = 64 if spec["long_dendrite"] else 8
    n = spec["n_cells"]
    n_cv = n * (1 + nd) + 32 * (1 + nd)
    n_conn = n * (min(fan_in, n - 1) + 1)
    slots = int((3.0 / spec["dt"] + 100) / max(1, min(64, int(round(3.0 / spec["dt"]))))) + 3
    return int(1.25 * (n_cv * 96 + n_conn * (72 + 16 * slots) + n * 256) + (8 << 20))


class _Resident:
    def __init__(self, spec, model, stream, n_cv, steps, start_s, reserved):
        self.spec, self.model, self.stream = spec, model, stream
        self.n_cv, self.steps, self.start_s = n_cv, steps, start_s
        self.reserved = reserved
        self.done_steps = 0
        self.event = None
        self.gid, self.step = [], []   # spikes drained after each quantum
        self.epoch_steps = model.info().epoch_steps

    def drain(self):
        g, st, _ = self.model.read_spikes()
        self.gid.append(g)
        self.step.append(st)


class Server:
    def __init__(self, hbm_budget_bytes: int = 64 << 30, quantum_cu: float = 1e6,
                 precision: int = E.PA_MIXED, device: int = 0, builders: int = 4,
                 max_resident: int = 512, build_threads: int = 1):
        import torch
        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.quantum_cu = quantum_cu
        self.precision = precision
        self.device = device
        self.max_resident = max_resident
        # host threads per model build (0: automatic); the builds overlap with
        # the scheduling loop that keeps the resident jobs' work launched
        self.build_threads = build_threads
        self.pool = ThreadPoolExecutor(max_workers=builders)
        torch.cuda.set_device(device)

    def _build(self, spec):
        torch = self.torch
        torch.cuda.set_device(self.device)
        net = W.serving_job(spec["n_cells"], spec["long_dendrite"], spec["dend_len_um"],
                            spec["dend_diam_um"], spec["seed"], dt=spec["dt"])
        stream = torch.cuda.Stream(device=self.device)
        m = E.Model(net, precision=self.precision, device=self.device,
                    stream=E.C.c_void_p(stream.cuda_stream),
                    flags=E.FLAG_BUILD_THREADS(self.build_threads))
        return net, m, stream

    def run(self, trace: List[dict], time_scale: float = 1.0) -> Dict:
        torch = self.torch
        pending = sorted(trace, key=lambda j: j["arrival_s"])
        qi = 0
        building = []          # (future, spec, reserved bytes)
        resident: List[_Resident] = []
        results: List[JobResult] = []
        used = 0
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        while qi < len(pending) or building or resident:
            t = now()
            # admit arrived jobs while the budget allows
            while qi < len(pending) and pending[qi]["arrival_s"] * time_scale <= t:
                spec = pending[qi]
                need = estimate_spec_bytes(spec)
                if used + need > self.budget or len(resident) + len(building) >= self.max_resident:
                    break
                used += need
                building.append((self.pool.submit(self._build, spec), spec, need))
                qi += 1
            # collect finished builds
            still = []
            for fut, spec, need in building:
                if fut.done():
                    net, m, stream = fut.result()
                    steps = int(round(spec["duration_ms"] / net.dt))
                    resident.append(_Resident(spec, m, stream, net.n_cv, steps, now(), need))
                else:
                    still.append((fut, spec, need))
            building = still
            # advance every resident job whose previous quantum has finished
            progressed = False
            finished = []
            for r in resident:
                if r.event is not None and not r.event.query():
                    continue
                if r.event is not None:
                    r.drain()             # the quantum is complete: stream its spikes out
                    r.event = None
                if r.done_steps >= r.steps:
                    finished.append(r)
                    continue
                # whole 8-epoch graph launches, about quantum_cu compartment-updates
                blk = 8 * r.epoch_steps
                q = blk * max(1, min(64, int(self.quantum_cu / (r.n_cv * blk))))
                r.done_steps = min(r.steps, r.done_steps + q)
                r.model.advance(r.done_steps * r.model.dt)
                r.event = torch.cuda.Event()
                r.event.record(r.stream)
                progressed = True
            for r in finished:
                r.drain()
                g, st = np.concatenate(r.gid), np.concatenate(r.step)
                w = r.model.read_weights()
                results.append(JobResult(r.spec["job_id"], r.spec["arrival_s"] * time_scale,
                                         r.start_s, now(), r.n_cv, r.steps, len(g),
                                         spike_digest(g, st), w))
                r.model.close()
                resident.remove(r)
                used -= r.reserved
            if not progressed and not finished:
                # nothing to do right now: wait for the next arrival or completion
                time.sleep(0.0005)
        wall = now()
        self.pool.shutdown(wait=True)
        lat = np.array([r.latency_s for r in results])
        cu = float(sum(r.n_cv * r.steps for r in results))
        first = min(j["arrival_s"] for j in trace) * time_scale
        return {"results": sorted(results, key=lambda r: r.job_id), "wall_s": wall,
                "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
                "cu": cu, "cu_per_s": cu / max(wall - first, 1e-9)}


def spike_digest(gid, step) -> int:
    return zlib.crc32(np.ascontiguousarray(step, np.int64).tobytes(),
                      zlib.crc32(np.ascontiguousarray(gid, np.int32).tobytes()))


def run_alone(spec, precision=E.PA_FP64, device=0, chunk_ms=1000.0):
    """One job by itself on the default stream (the comparison path); spikes are
    read back every chunk_ms of simulated time."""
    net = W.serving_job(spec["n_cells"], spec["long_dendrite"], spec["dend_len_um"],
                        spec["dend_diam_um"], spec["seed"], dt=spec["dt"])
    m = E.Model(net, precision=precision, device=device)
    steps = int(round(spec["duration_ms"] / net.dt))
    per = max(1, int(round(chunk_ms / net.dt)))
    gs, ss = [], []
    done = 0
    while done < steps:
        done = min(steps, done + per)
        m.advance(done * net.dt)
        g, s, _ = m.read_spikes()
        gs.append(g)
        ss.append(s)
    w = m.read_weights()
    m.close()
    return net.n_cv, steps, np.concatenate(gs), np.concatenate(ss), w
