"""Continuous-batching simulation server on one GPU.

Jobs (one network each) arrive over time.  The server admits a job as soon as
the HBM budget allows, builds it on a background thread (pa_build_model, on
the job's own stream), and keeps its state resident.  Every resident job is a
member of one batch (pa_batch_*): each min-delay epoch of all resident jobs is
ONE launch of the time-step kernel over every job's cell groups, with each
job's Poisson draws, routing and spike record on parallel branches, replayed
from CUDA graphs (8 epochs per graph launch) that are captured again when the
membership changes.  New jobs join at epoch boundaries between ticks (a tick
is `epochs_per_tick` epochs); a job with fewer whole epochs left than a tick
leaves the batch and finishes alone (its last epochs and partial epoch on
direct launches).  Spikes are drained about every `drain_ms` of a job's
simulated time; a finished job's spikes and weights are read back and its
memory freed, which makes room for waiting jobs.  Latency is measured from a
job's arrival to the moment its results are on the host.

All jobs of the serving trace share dt (0.2 ms), the 3 ms delay (15-step
epochs), the precision and the tree class (ball-and-stick chains), so one
batch holds them all.  Jobs never share device state, and a batch member
takes exactly the steps it takes alone, so a job's results are the same alone
and in the mix, bit for bit; tests/test_serving.py checks this.
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
    def __init__(self, spec, model, n_cv, steps, start_s, reserved):
        self.spec, self.model = spec, model
        self.n_cv, self.steps, self.start_s = n_cv, steps, start_s
        self.reserved = reserved
        self.epoch_steps = model.info().epoch_steps
        self.gid, self.step = [], []
        self.last_drain = 0

    def drain(self):
        g, st, _ = self.model.read_spikes()
        self.gid.append(g)
        self.step.append(st)
        self.last_drain = self.model.step


class Server:
    def __init__(self, hbm_budget_bytes: int = 64 << 30, epochs_per_tick: int = 8,
                 precision: int = E.PA_MIXED, device: int = 0, builders: int = 4,
                 max_resident: int = 512, build_threads: int = 1, drain_ms: float = 1000.0):
        import torch
        self.torch = torch
        self.budget = int(hbm_budget_bytes)
        self.tick = max(1, int(epochs_per_tick))
        self.precision = precision
        self.device = device
        self.max_resident = max_resident
        self.drain_ms = drain_ms
        # host threads per model build; the builds overlap with the loop that
        # keeps the batch's work launched
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
                    flags=E.FLAG_NARROW_ONLY | E.FLAG_BUILD_THREADS(self.build_threads))
        m._build_stream = stream           # keep the stream alive until the model moves
        return net, m

    def run(self, trace: List[dict], time_scale: float = 1.0) -> Dict:
        torch = self.torch
        stream = torch.cuda.Stream(device=self.device)
        batch = E.Batch(self.device, stream=E.C.c_void_p(stream.cuda_stream))
        pending = sorted(trace, key=lambda j: j["arrival_s"])
        qi = 0
        building = []          # (future, spec, reserved bytes)
        members: List[_Resident] = []
        results: List[JobResult] = []
        used = 0
        ticks = member_ticks = 0
        host_advance = 0.0
        tick_log = []          # (event after the tick, compartment-updates of the tick)
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0

        def finish(r):
            m = r.model
            m.advance(r.steps * m.dt)          # the last epochs alone (direct launches)
            r.drain()
            g, st = np.concatenate(r.gid), np.concatenate(r.step)
            w = m.read_weights()
            results.append(JobResult(r.spec["job_id"], r.spec["arrival_s"] * time_scale,
                                     r.start_s, now(), r.n_cv, r.steps, len(g),
                                     spike_digest(g, st), w))
            m.close()
            return r.reserved

        while qi < len(pending) or building or members:
            t = now()
            # admit arrived jobs while the budget allows
            while qi < len(pending) and pending[qi]["arrival_s"] * time_scale <= t:
                spec = pending[qi]
                need = estimate_spec_bytes(spec)
                if used + need > self.budget or len(members) + len(building) >= self.max_resident:
                    break
                used += need
                building.append((self.pool.submit(self._build, spec), spec, need))
                qi += 1
            # finished builds join the batch (at step 0, an epoch boundary)
            still = []
            for fut, spec, need in building:
                if fut.done():
                    net, m = fut.result()
                    steps = int(round(spec["duration_ms"] / net.dt))
                    r = _Resident(spec, m, net.n_cv, steps, now(), need)
                    if steps >= self.tick * r.epoch_steps:
                        batch.add(m)
                        members.append(r)
                    else:
                        used -= finish(r)      # shorter than one tick: runs alone
                else:
                    still.append((fut, spec, need))
            building = still
            if not members:
                if qi < len(pending) or building:
                    time.sleep(0.0005)
                continue
            # one tick: every member advances `tick` epochs in grouped launches
            ta = time.perf_counter()
            batch.advance_epochs(self.tick)
            host_advance += time.perf_counter() - ta
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            tick_log.append((ev, sum(r.n_cv * self.tick * r.epoch_steps for r in members)))
            ticks += 1
            member_ticks += len(members)
            done = []
            for r in members:
                left = r.steps - r.model.step
                if left < self.tick * r.epoch_steps:
                    done.append(r)
                elif (r.model.step - r.last_drain) * r.model.dt >= self.drain_ms:
                    r.drain()
            for r in done:
                batch.remove(r.model)
                members.remove(r)
                used -= finish(r)
        wall = now()
        binfo = batch.info()
        batch.close()
        # the batch's device-side rate: the most compartment-updates of grouped
        # ticks completed within any one second (events on the batch's stream)
        peak = 0.0
        if len(tick_log) > 1:
            torch.cuda.synchronize(self.device)
            t = np.array([tick_log[0][0].elapsed_time(e) for e, _ in tick_log]) * 1e-3
            c = np.cumsum([cu_t for _, cu_t in tick_log])
            span = t[-1] - t[0]
            win = min(1.0, span) if span > 0 else 0.0
            if win > 0:
                j = np.searchsorted(t, t - win, side="left")
                peak = float(np.max((c - np.where(j > 0, c[np.maximum(j - 1, 0)], 0.0)) / win))
        self.pool.shutdown(wait=True)
        lat = np.array([r.latency_s for r in results])
        cu = float(sum(r.n_cv * r.steps for r in results))
        first = min(j["arrival_s"] for j in trace) * time_scale
        return {"results": sorted(results, key=lambda r: r.job_id), "wall_s": wall,
                "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
                "cu": cu, "cu_per_s": cu / max(wall - first, 1e-9),
                "graph_launches": binfo["graph_launches"], "graph_captures": binfo["captures"],
                "ticks": ticks, "mean_members_per_tick": member_ticks / max(ticks, 1),
                "peak_1s_cu_per_s": peak,
                "host_s_in_batch_advance": host_advance}


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
