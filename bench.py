#!/usr/bin/env python3
"""Benchmark of the plastic multi-compartment time-step loop on B300.

Workload: the large mixed-precision network -- 100,000 HH-soma cells on random
binary dendritic trees of 51-501 CVs (each cell's tree drawn from a seeded pool
of 4,096 random trees), 10^7 pair-STDP synapses (fan-in 100, delays 1-5 ms),
2 Hz Poisson drive, dt = 0.025 ms.  One benchmark step is one min-delay epoch
(40 time steps = 1 ms) of the whole loop: Poisson drive, synaptic and
mechanism updates, cable assembly + Hines solve, detection, CSR routing.

value = compartment-updates/s (CU/s = CVs x time steps / device time) of the
mixed-precision path; the FP64 path is timed on the same GPU and reported
beside it.  All inputs are synthetic and resident in HBM before timing; the
working set (several GB) is far larger than the 126 MB L2, so no L2 flush is
needed between steps.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compartment-updates/s, mixed vs FP64 plain, same GPU; serving p50/p99 latency"
UNIT = "CU/s"
N_SM = 148
DFMA_PER_SM_CLK = 2            # nominal FP64 FMA lanes per SM and clock (context only)
RCP64_DFMA_EQ = 465.0 / 71.0   # measured: FP64 FMA 465 G/s vs FP64 reciprocal 71 G/s on B300
FALLBACK_HBM_GBS = 6400.0      # the profiling recipe's fallback when no measured peak exists
# The survey's algorithmic bytes per compartment-update for the large STDP
# network (hot-path scope table, measurement row): FP64 about 60 B/CU (V read
# and write 16, axial coefficient 8, parent 4, C/dt 8, leak 8 per CV; HH gates
# per soma; synapse state amortised at about 0.36 synapses per CV), mixed about
# 45 B/CU (FP32 mechanism state and FP32-stored geometry).
SURVEY_BYTES_PER_CU = {"fp64": 60.0, "mixed": 45.0, "fp32": 45.0}
# DRAM bytes per compartment-update of the epoch kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of a 65,536-cell launch of the
# same generator, shape 0, the kernels for reversal potentials of +0: 82.47 GB
# (mixed, float-float solve, leak E-term formed) and 88.42 GB (FP64) for
# 735.3 M CU), scaled to a full launch by the CUs it processes, since traffic
# grows in proportion to them; absent once the kernel has changed since the
# counters were taken (and for the FP32-mechanism kernel, not captured).
TRAFFIC_B_PER_CU = {"mixed": 112.2, "fp64": 120.2}


def measured_peaks():
    """MEASURED_PEAKS.json (written by the pool's driver): HBM copy bandwidth."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "of measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "of fallback (no MEASURED_PEAKS.json)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=40)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--cells", type=int, default=100_000)
    p.add_argument("--shapes", type=int, default=4096)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--precision", default="all", choices=["all", "both", "mixed", "fp64", "fp32"],
                   help="all: mixed (the headline), fp64 and fp32; both: mixed and fp64")
    p.add_argument("--busyring", action="store_true",
                   help="run the paper's busyring table instead (setup and propagation)")
    p.add_argument("--busyring-cells", default="1024,16384,32768")
    p.add_argument("--busyring-depths", default="0,2,10")
    p.add_argument("--busyring-flags", type=int, default=0,
                   help="extra pa_options flags for the busyring models (e.g. cell bins)")
    p.add_argument("--no-batched", action="store_true",
                   help="skip the batched morphology-sweep measurement")
    p.add_argument("--only-batched", action="store_true",
                   help="run only the batched morphology-sweep measurement")
    p.add_argument("--batched-epochs", type=int, default=200)
    p.add_argument("--serve-jobs", type=int, default=80,
                   help="serving measurement on this many jobs of the trace (0: skip)")
    p.add_argument("--serve-no-alone", action="store_true",
                   help="skip the serving baseline (every job alone on the FP64 path)")
    p.add_argument("--recall", action="store_true",
                   help="time the 10s-recall and 8h-recall paradigms of the tagging-and-capture "
                        "networks (ball-and-stick with a PRP pool; 48-CV cells with PRP diffusion)")
    p.add_argument("--shape", type=int, default=-1,
                   help="force this epoch-kernel shape instead of autotuning")
    return p.parse_args()


def workload(n_cells, n_shapes, seed_offset=0):
    from paper_2411_16445_b300 import workloads as W
    net = W.large_stdp(n_cells=n_cells, n_shapes=n_shapes)
    if seed_offset:
        net.seed = (net.seed + 0x9E3779B97F4A7C15 * seed_offset) & (2**64 - 1)
    return net


def net_stats(net):
    ncv = net.cell_ncv()
    kinds = net.mech_kind[net.conn_mech]
    # rows that carry a first child (i + 1 with parent i) and non-first children
    first = np.array([int(np.sum(m.parent[1:] == np.arange(m.n_cv - 1))) for m in net.morphs])
    other = np.array([m.n_cv - 1 for m in net.morphs]) - first
    per_cell = np.bincount(net.cell_morph, minlength=len(net.morphs))
    return {
        "n_cells": int(net.n_cells),
        "n_cv": int(ncv.sum()),
        "n_syn": int(net.n_conn),
        "n_stdp": int(np.sum(kinds == 13)),
        "n_expsyn": int(np.sum(kinds == 10)),
        "n_first": int(np.dot(per_cell, first)),
        "n_other": int(np.dot(per_cell, other)),
        "tree": any(not m.is_chain() for m in net.morphs),
        # every synaptic reversal potential exactly +0 (the kernels' es_zero case)
        "es_zero": all(np.float64(net.mech_params[m][1]).tobytes() == bytes(8)
                       for m in np.unique(net.conn_mech) if net.mech_kind[m] in (10, 11, 12, 13)),
    }


def per_cu_model(st, prec):
    """Work of one compartment-update of this engine's layout, amortising soma and
    synapse work (prec: "fp64", "mixed" or "fp32").
    Bytes: state that must stream every step (V read+write, four FP64 cable
    coefficients: C/dt, diagonal, leak E term, axial coupling; 2-byte parent
    index on trees) plus per-synapse state read+write (the conductance: 8 B in
    FP64 and in mixed, where it is a float-float pair; 4 B in FP32; the STDP
    traces are touched only at events), CV index and event word.
    FP64 ops (FMA, multiply or add; the FP64 pipe's work): per row the diagonal
    and right-hand-side assembly (3: d + g_syn, C/dt V + E-term, + gE_syn), the
    f and x' products (2) and the back substitution (1); two FMAs per child
    eliminated into its parent (carried first child or other child); HH per
    soma; 4 per synapse in FP64 (decay, two sums, g E), 0 in FP32.  When every
    reversal potential is +0 the g E terms are signed zeros handled on the
    integer pipes: one assembly addition per row and the g E product and sum
    per synapse drop out.  In mixed the conductances, per-CV sums and the row
    itself (assembly, elimination, back substitution) are float-float on the
    FP32 pipes: only HH remains on the FP64 pipe.  The FP64 row reciprocal runs
    on the integer pipes (correctly rounded, about forty integer ops) and is
    not counted."""
    gb = 4 if prec == "fp32" else 8
    cv_bytes = 16 + 32 + (2 if st["tree"] else 0)
    syn_b = 2 * gb + 4 + 8
    syn_bytes = (st["n_stdp"] + st["n_expsyn"]) * syn_b
    bytes_per_cu = cv_bytes + syn_bytes / st["n_cv"]
    ez = st.get("es_zero", False)
    solve = (5 if ez else 6) * st["n_cv"] + 2 * (st["n_first"] + st["n_other"])
    if prec == "mixed":
        solve = 0
    hh = 153 + 6 * RCP64_DFMA_EQ + 20                  # 9 model exps, 6 divisions, currents
    per_syn = {"fp64": 2 if ez else 4, "mixed": 0, "fp32": 0}[prec]
    syn = per_syn * (st["n_stdp"] + st["n_expsyn"])
    fp64_per_cu = (solve + hh * st["n_cells"] + syn) / st["n_cv"]
    return bytes_per_cu, fp64_per_cu


class ClockSampler:
    def __init__(self, device):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(device)],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_total(ms_local, cu_per_rank, ws, device=None):
    """Replicas (one independent network per rank, no data-path collective): the
    job's time is the slowest rank's, and the job processed ws x cu_per_rank
    compartment-updates.  Returns (max ms over ranks, whole-job CU/s)."""
    ms = ms_local
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_local], dtype=torch.float64,
                         device=f"cuda:{device}" if device is not None else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, cu_per_rank * ws / (ms * 1e-3)


def model_flags(args):
    from paper_2411_16445_b300 import engine as E
    f = E.FLAG_TIME_KERNELS
    f |= E.flag_shape(args.shape) if args.shape >= 0 else E.FLAG_AUTOTUNE
    return f


def time_gpu(net, precision, steps, warmup, device, stream_barrier, flags):
    import torch
    from paper_2411_16445_b300 import engine as E
    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream(device)
    t0 = time.perf_counter()
    m = E.Model(net, precision=precision, device=device, stream=E.C.c_void_p(stream.cuda_stream),
                flags=flags)
    setup_s = time.perf_counter() - t0
    info = m.info()
    shape, trial_ms = m.tuning()
    E_steps = info.epoch_steps
    m.advance(warmup * E_steps * net.dt)
    m.sync()
    m.read_spikes()
    m.reset_kernel_stats()
    stream_barrier()
    torch.cuda.synchronize(device)
    sampler = ClockSampler(device)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    m.advance((warmup + steps) * E_steps * net.dt)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize(device)
    clocks = sampler.stop()
    stream_barrier()
    ms = ev0.elapsed_time(ev1)
    m.sync()
    ks = m.kernel_stats()
    gid, _, _ = m.read_spikes()
    res = {"ms": ms, "epoch_steps": E_steps, "n_cv": info.n_cv, "setup_s": setup_s,
           "epoch_kernel_ms": ks.epoch_kernel_ms, "event_kernels_ms": ks.event_kernels_ms,
           "epoch_launches": ks.epoch_launches, "kernel_launches": ks.kernel_launches,
           "spikes": int(len(gid)), "device_bytes": info.device_bytes, "clocks": clocks,
           "shape": shape, "shape_trial_ms": [round(float(x), 3) for x in trial_ms]}
    m.close()
    return res


def time_e2e(net, precision, steps, device):
    """The user's end-to-end path through the C-ABI: descriptors from host memory
    uploaded by pa_build_model, pa_advance one epoch at a time with the epoch's
    spikes read back to the host each time, final weights read back."""
    import torch
    from paper_2411_16445_b300 import engine as E
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    m = E.Model(net, precision=precision, device=device)   # the default call: no autotuning
    info = m.info()
    h2d = info.device_bytes
    spikes = 0
    for s in range(steps):
        m.advance((s + 1) * info.epoch_steps * net.dt)
        g, _, _ = m.read_spikes()
        spikes += len(g)
    w = m.read_weights()
    torch.cuda.synchronize(device)
    t = time.perf_counter() - t0
    m.close()
    cu = info.n_cv * info.epoch_steps * steps
    d2h = spikes * (4 + 8 + 8) + w.nbytes
    return {"value": cu / t, "unit": UNIT, "h2d_bytes_per_step": int(h2d / steps),
            "d2h_bytes_per_step": int(d2h / steps), "wall_s": t,
            "note": "includes pa_build_model with default flags (host descriptors -> HBM, "
                    "no autotuning) and per-epoch spike read-back"}


def oracle_sample(n_cells, n_shapes, budget_s=12.0, max_steps=40000, warm=2):
    """The FP64 CPU oracle on a bounded sample of the workload: the same generator
    at n_cells cells, timed over whole steps until the CPU budget is spent."""
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle as O
    net = workload(n_cells, n_shapes)
    o = O.Oracle(net)
    o.run(warm)
    n_cv = net.n_cv
    done, t = 0, 0.0
    chunk = 5
    while t < budget_s and done < max_steps:
        t0 = time.perf_counter()
        o.run(chunk)
        t += time.perf_counter() - t0
        done += chunk
    return {"value": n_cv * done / t, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle", "sample": f"{n_cells} cells ({n_cv} CVs, {net.n_conn} synapses) of "
            f"the same generator, {done} time steps, FP64, OpenMP over cells", "seconds": t}


def serving_bench(n_jobs, device, alone=True, load=0.7):
    """Continuous-batching server on the first n_jobs of the seeded serving trace
    (Poisson arrivals at 20 jobs/s, sizes log-uniform 1-20000 cells, durations
    log-uniform 0.1-10 s, dt 0.2 ms), mixed precision, jobs admitted by HBM
    budget and advanced together as one batch (one grouped time-step launch per
    epoch for all resident jobs).
      1. capacity: every job submitted at t = 0; the batch's device-side rate
         (the most compartment-updates completed within one second);
      2. paced: the same jobs with their arrival times stretched so that the
         offered load is `load` x that capacity; p50 / p99 latency from arrival
         to results on the host.
    Baseline: every job alone on the plain FP64 path (build, run, read back),
    served one at a time in arrival order of the paced run; its latencies
    follow from the measured per-job times."""
    import torch
    from paper_2411_16445_b300 import engine as E
    from paper_2411_16445_b300 import serving as S
    from paper_2411_16445_b300 import workloads as W
    trace = W.serving_trace()[:n_jobs]
    keys = ("graph_launches", "graph_captures", "ticks", "mean_members_per_tick",
            "host_s_in_batch_advance", "peak_1s_cu_per_s")
    sat = S.Server(hbm_budget_bytes=64 << 30, precision=E.PA_MIXED, device=device).run(
        trace, time_scale=0.0)
    cu = sat["cu"]
    capacity = sat["peak_1s_cu_per_s"]
    span = trace[-1]["arrival_s"] - trace[0]["arrival_s"]
    offered_1 = cu / max(span, 1e-9)
    scale = max(1.0, offered_1 / max(load * capacity, 1e-9))
    out = S.Server(hbm_budget_bytes=64 << 30, precision=E.PA_MIXED, device=device).run(
        trace, time_scale=scale)
    res = {"jobs": n_jobs, "precision": "mixed",
           "sample": f"first {n_jobs} jobs of the 2000-job seeded trace "
                     f"({span:.1f} s of arrivals at 20 jobs/s)",
           "capacity_cu_per_s": capacity,
           "capacity_note": "all jobs submitted at t = 0; the batch's device-side rate, the "
                            "most compartment-updates its grouped ticks completed in one second",
           "saturated": {"wall_s": sat["wall_s"], "cu_per_s": sat["cu_per_s"],
                         "server": {k: sat[k] for k in keys}},
           "arrival_time_scale": scale,
           "offered_cu_per_s": offered_1 / scale,
           "offered_cu_per_s_unscaled": offered_1,
           "p50_s": out["p50_s"], "p99_s": out["p99_s"], "cu": cu,
           "cu_per_s": out["cu_per_s"], "wall_s": out["wall_s"],
           "server": {k: out[k] for k in keys},
           "hbm_budget_bytes": 64 << 30,
           "launch": "all resident jobs in one batch: one grouped time-step launch per epoch, "
                     "8 epochs per CUDA-graph launch, recaptured on membership changes"}
    if not alone:
        return res
    t_alone = []
    for spec in trace:
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        S.run_alone(spec, precision=E.PA_FP64, device=device)
        torch.cuda.synchronize(device)
        t_alone.append(time.perf_counter() - t0)
    free_at, lat = 0.0, []
    for spec, t in zip(trace, t_alone):
        start = max(spec["arrival_s"] * scale, free_at)
        free_at = start + t
        lat.append(free_at - spec["arrival_s"] * scale)
    lat = np.array(lat)
    first = trace[0]["arrival_s"] * scale
    res["alone_fp64"] = {"p50_s": float(np.percentile(lat, 50)),
                         "p99_s": float(np.percentile(lat, 99)),
                         "cu_per_s": cu / max(free_at - first, 1e-9),
                         "busy_s": float(sum(t_alone)),
                         "note": "each job built, run and read back alone on the FP64 path; "
                                 "jobs served one at a time in the paced arrival order"}
    return res


def batched_bench(device, epochs=200, warmup=8):
    """Many networks in one persistent launch per min-delay epoch: the batched
    morphology sweep (64 independent 500-cell ball-and-stick networks with
    4-64-CV dendrites, calcium-plastic synapses, dt 0.2 ms), every epoch a
    CUDA-graph launch, kernel shape autotuned.  Mixed and FP64; one network
    alone (same generator, one network) for comparison."""
    import torch
    from paper_2411_16445_b300 import engine as E
    from paper_2411_16445_b300 import workloads as W
    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream(device)

    def run(net, prec):
        m = E.Model(net, precision=prec, device=device, stream=E.C.c_void_p(stream.cuda_stream),
                    flags=E.FLAG_AUTOTUNE)
        info = m.info()
        Es = info.epoch_steps
        m.advance(warmup * Es * net.dt)
        m.read_spikes()
        torch.cuda.synchronize(device)
        m.reset_kernel_stats()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        m.advance((warmup + epochs) * Es * net.dt)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        ks = m.kernel_stats()
        m.read_spikes()
        res = {"cu_per_s": info.n_cv * Es * epochs / (ms * 1e-3), "ms_per_epoch": ms / epochs,
               "graph_launches": ks.graph_launches, "kernel_launches": ks.kernel_launches,
               "shape": m.tuning()[0]}
        m.close()
        return res, info

    net = W.morphology_sweep()
    mixed, info = run(net, E.PA_MIXED)
    fp64, _ = run(net, E.PA_FP64)
    fp32, _ = run(net, E.PA_FP32)
    one, _ = run(W.morphology_sweep(n_nets=1), E.PA_MIXED)
    return {"workload": "morphology_sweep", "n_networks": 64, "n_cells": info.n_cells,
            "n_cv": info.n_cv, "dt_ms": net.dt, "epoch_steps": info.epoch_steps,
            "epochs_timed": epochs, "launch": "one persistent epoch kernel per min-delay epoch "
            "for all 64 networks, whole epochs as CUDA-graph launches (8 epochs per launch)",
            "mixed": mixed, "fp64": fp64, "fp32": fp32, "one_network_alone_mixed": one}


# The paper's busyring propagation times [s] (Table 8: CPU, Arbor with SIMD on a
# 64-core Threadripper PRO 5995WX; Table 9: the same with an NVIDIA T1000), keyed
# by (cells, depth, stdp): (cpu, cpu + gpu).
PAPER_BUSYRING = {
    (1024, 0, False): (0.19, 0.30), (1024, 2, False): (0.28, 0.41), (1024, 10, False): (2.48, 2.99),
    (1024, 0, True): (0.68, 0.78), (1024, 2, True): (0.79, 1.00), (1024, 10, True): (3.01, 3.50),
    (16384, 0, False): (2.86, 2.81), (16384, 2, False): (4.23, 4.15), (16384, 10, False): (40.72, 40.45),
    (16384, 0, True): (10.61, 10.44), (16384, 2, True): (12.37, 12.04), (16384, 10, True): (49.90, 49.05),
    (32768, 0, False): (5.31, 5.30), (32768, 2, False): (7.86, 7.78), (32768, 10, False): (81.09, 80.44),
    (32768, 0, True): (21.00, 20.47), (32768, 2, True): (24.45, 23.71), (32768, 10, True): (99.60, 97.75),
}


def busyring_bench(device, cells_list, depths, precision_name, extra_flags=0):
    """The busyring benchmark at the paper's sizes: 200 ms at dt 0.025 ms, setup
    (network description -> resident model) and propagation (pa_advance over the
    whole run, CUDA events on the model's stream) timed separately, as in
    Tables 8-9; trees from a seeded pool of 4096 shapes above 4096 cells."""
    import torch
    from paper_2411_16445_b300 import engine as E
    from paper_2411_16445_b300 import workloads as W
    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream(device)
    prec = {"mixed": E.PA_MIXED, "fp32": E.PA_FP32}.get(precision_name, E.PA_FP64)
    rows = []
    for n in cells_list:
        for d in depths:
            for stdp in (False, True):
                net = W.busyring(n_cells=n, depth=d, stdp=stdp,
                                 n_shapes=4096 if n > 4096 else None)
                torch.cuda.synchronize(device)
                t0 = time.perf_counter()
                m = E.Model(net, precision=prec, device=device,
                            stream=E.C.c_void_p(stream.cuda_stream),
                            flags=E.FLAG_AUTOTUNE | extra_flags)
                torch.cuda.synchronize(device)
                setup = time.perf_counter() - t0
                info = m.info()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                steps = int(round(200.0 / net.dt))
                e0.record(stream)
                m.advance(steps * net.dt)
                e1.record(stream)
                e1.synchronize()
                prop = e0.elapsed_time(e1) * 1e-3
                g, _, _ = m.read_spikes()
                m.close()
                paper = PAPER_BUSYRING.get((n, d, stdp))
                rows.append({"cells": n, "depth": d, "stdp": stdp, "n_cv": info.n_cv,
                             "wide_cells": info.n_wide,
                             "synapses": net.n_conn, "setup_s": round(setup, 3),
                             "propagation_s": round(prop, 4),
                             "cu_per_s": info.n_cv * steps / prop, "spikes": int(len(g)),
                             "paper_propagation_s_cpu": paper[0] if paper else None,
                             "paper_propagation_s_cpu_gpu": paper[1] if paper else None,
                             "speedup_vs_paper_cpu": paper[0] / prop if paper else None})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    return rows


def _with_step(net, cells, i_nA, t_on, t_off):
    """a copy of net whose cells `cells` receive a somatic current step"""
    import copy
    n2 = copy.copy(net)
    n2.cell_istep = net.cell_istep.copy()
    n2.cell_ton = net.cell_ton.copy()
    n2.cell_toff = net.cell_toff.copy()
    n2.cell_istep[cells] = i_nA
    n2.cell_ton[cells] = t_on
    n2.cell_toff[cells] = t_off
    return n2


def recall_bench(device, n_long_per_hour=3600, cpu=True):
    """The '10s-recall' and '8h-recall' paradigms of the tagging-and-capture
    network (Secs. on memory consolidation, Fig. 6 and Supplementary Fig. S13):
    2000 cells (1600 E + 400 I), learning by a 0.1 s current step into a core
    of 150 E cells, recall by a 0.1 s step into 75 of them, 10 s or 8 h later.
    The recall stimulus lives in a second model into which the whole state is
    swapped (the paradigm's state-saving mechanism); the 8 h wait is a
    fast-forward of the slow plasticity variables in long steps
    (n_long_per_hour per hour).  Networks: ball-and-stick cells (9 CVs) with
    one PRP pool per cell, and the 48-CV morphological cells of Table 6 (small
    cells, large dendrites) with PRP diffusing at 1e-11 m2/s; the first again
    with the plasticity noise of Table 5 (sigma_pl = 2.90436 mV; 10s-recall
    only), for the cost of the noise.  FP64; wall times of each phase
    (synchronised), as the paper's totals."""
    import torch
    from paper_2411_16445_b300 import engine as E
    from paper_2411_16445_b300 import workloads as W
    torch.cuda.set_device(device)
    stream = E.C.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    nets = {
        "ball_and_stick_pool": W.recurrent_stc(n_exc=1600, n_inh=400),
        "morpho48_diffusion": W.recurrent_stc_morpho(n_exc=1600, n_inh=400, d_p=1e-2,
                                                     large_dend=True),
        # the same pool network with Table 5's plasticity noise (10s-recall only)
        "ball_and_stick_pool_noise": W.recurrent_stc(n_exc=1600, n_inh=400,
                                                     sigma_pl=2.90436),
    }
    core = np.arange(150)
    t_learn = (100.0, 200.0)
    rows = []
    for name, base in nets.items():
        dt = base.dt
        learn = _with_step(base, core, 1.0, *t_learn)
        fields = [E.FIELD_V, E.FIELD_GATES, E.FIELD_PRP, E.FIELD_G, E.FIELD_C, E.FIELD_H,
                  E.FIELD_Z]
        paradigms = (("10s-recall", 10_000.0), ("8h-recall", 8 * 3600e3))
        for paradigm, wait_ms in paradigms[:1] if name.endswith("noise") else paradigms:
            t_swap = t_learn[1] + wait_ms
            recall = _with_step(base, core[:75], 1.0, t_swap, t_swap + 100.0)
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            a = E.Model(learn, precision=E.PA_FP64, device=device, stream=stream)
            torch.cuda.synchronize(device)
            t1 = time.perf_counter()
            t_full = t_learn[1] + min(wait_ms, 10_000.0)      # full dynamics after learning
            a.advance(t_full)
            a.sync()
            t2 = time.perf_counter()
            n_long = 0
            if wait_ms > 10_000.0:
                n_long = int(round((t_swap - t_full) / 3600e3 * n_long_per_hour))
                a.fast_forward(t_swap - t_full, n_long)
                a.sync()
            t3 = time.perf_counter()
            fl = fields + ([E.FIELD_PRP_CV] if name.endswith("diffusion") else [])
            saved = {f: a.read_state(f) for f in fl}
            a.close()
            b = E.Model(recall, precision=E.PA_FP64, device=device, stream=stream)
            b.fast_forward(t_swap, 1)                          # the clock; state overwritten
            for f in fl:
                if f != E.FIELD_PRP or not name.endswith("diffusion"):
                    b.write_state(f, saved[f])
            b.sync()
            t4 = time.perf_counter()
            b.advance(t_swap + 300.0)
            g, _, _ = b.read_spikes()
            b.sync()
            t5 = time.perf_counter()
            info = b.info()
            full_steps = int(round(t_full / dt)) + int(round(300.0 / dt))
            rows.append({"network": name, "paradigm": paradigm, "n_cells": base.n_cells,
                         "n_cv": int(info.n_cv), "dt_ms": dt, "full_steps": full_steps,
                         "long_steps": n_long, "setup_s": round(t1 - t0, 3),
                         "learn_and_wait_s": round(t2 - t1, 3), "fast_forward_s": round(t3 - t2, 4),
                         "state_swap_s": round(t4 - t3, 3), "recall_s": round(t5 - t4, 3),
                         "total_s": round(t5 - t0, 3),
                         "cu_per_s_full": info.n_cv * full_steps / ((t2 - t1) + (t5 - t4)),
                         "recall_spikes": int(len(g))})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    out = {"benchmark": "recall_paradigms", "precision": "fp64", "rows": rows}
    if cpu:
        # the oracle on the host cores: the full-dynamics part of the 10s-recall
        # of each network, timed over a bounded sample of steps
        import oracle as O
        cores = os.cpu_count() or 1
        os.environ.setdefault("OMP_NUM_THREADS", str(cores))
        ref = {}
        for name, base in nets.items():
            if name.endswith("noise"):
                continue
            o = O.Oracle(_with_step(base, core, 1.0, *t_learn))
            t0 = time.perf_counter()
            k = 5000
            o.run(k)
            t = time.perf_counter() - t0
            ref[name] = {"cu_per_s": base.n_cv * k / t, "steps_timed": k,
                         "est_10s_recall_full_s": t / k * (int(round(10_500.0 / base.dt)))}
        out["cpu_oracle"] = {"cores": int(os.environ["OMP_NUM_THREADS"]), "networks": ref}
    return out


def reference_arm(args):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    import oracle as O
    n_cells = min(args.cells, 4096)
    net = workload(n_cells, min(args.shapes, n_cells))
    o = O.Oracle(net)
    steps_per_sample = 4
    o.run(args.warmup * steps_per_sample)
    t0 = time.perf_counter()
    o.run(args.steps * steps_per_sample)
    t = time.perf_counter() - t0
    val = net.n_cv * steps_per_sample * args.steps / t
    sample = (f"each step: {steps_per_sample} time steps of {n_cells} cells ({net.n_cv} CVs) "
              f"of the large STDP network generator, FP64 oracle, OpenMP over cells")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "large_stdp", "n_cells": n_cells, "dt_ms": net.dt,
                       "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    # the serving measurement drives many streams at once
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.busyring:
        cells = [int(x) for x in args.busyring_cells.split(",")]
        rows = busyring_bench(0, cells, [int(x) for x in args.busyring_depths.split(",")],
                              args.precision if args.precision not in ("all", "both") else "fp64",
                              args.busyring_flags)
        print(json.dumps({"benchmark": "busyring", "unit": UNIT, "simulated_ms": 200.0,
                          "dt_ms": 0.025, "rows": rows,
                          "paper_hardware": "AMD Threadripper PRO 5995WX (64 cores), "
                                            "+ NVIDIA T1000 8GB for the cpu_gpu column"}),
              flush=True)
        return
    if args.recall:
        print(json.dumps(recall_bench(0, cpu=not args.no_cpu)), flush=True)
        return
    if args.only_batched:
        print(json.dumps({"batched": batched_bench(0, epochs=args.batched_epochs)}), flush=True)
        return
    import torch
    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

        def barrier():
            dist.barrier()
    else:
        def barrier():
            pass
    device = local
    net = workload(args.cells, args.shapes, seed_offset=rank)
    st = net_stats(net)
    runs = {}
    precs = {"mixed": 1, "fp64": 0, "fp32": 2}
    order = {"all": ["mixed", "fp64", "fp32"], "both": ["mixed", "fp64"]}.get(
        args.precision, [args.precision])
    for name in order:
        runs[name] = time_gpu(net, precs[name], args.steps, args.warmup, device, barrier,
                              model_flags(args))
    head = order[0]
    r = runs[head]
    ms = r["ms"]
    cu_per_rank = r["n_cv"] * r["epoch_steps"] * args.steps
    ms, value = replica_total(ms, cu_per_rank, ws, device)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return

    hbm_peak, hbm_note = measured_peaks()
    from paper_2411_16445_b300 import engine as E
    fma_rate = E.measure_fp64(device)["fma_per_s"]       # FP64 FMA/s, measured here

    def roofline(run, prec):
        """Top level: the epoch kernel against the HBM roof on the survey's algorithmic
        bytes; beside it the FP64 pipe, the engine's own layout bytes and the DRAM
        traffic ncu counted."""
        bpc, fpc = per_cu_model(st, prec)
        sbpc = SURVEY_BYTES_PER_CU[prec]
        cu_launch = run["n_cv"] * run["epoch_steps"]
        t_launch = run["epoch_kernel_ms"] / max(run["epoch_launches"], 1) * 1e-3
        ach_gbs = sbpc * cu_launch / t_launch / 1e9
        clk = (run["clocks"] or {}).get("sm_mhz") or 2032.0
        fp64_peak = 2 * fma_rate / 1e12
        fp64_ach = 2 * fpc * cu_launch / t_launch / 1e12
        tb = TRAFFIC_B_PER_CU.get(prec)
        return {"bound": "hbm", "achieved": ach_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach_gbs / hbm_peak, "traffic": tb * cu_launch if tb else None,
                "kernel": "epoch_kernel", "peak_note": hbm_note,
                "algorithmic_bytes_per_cu": sbpc,
                "algorithmic_note": "the survey's per-CU bytes for this network "
                                    "(hot-path scope table, measurement row) x CVs x steps of "
                                    "one launch / the launch's mean device time (CUDA events)",
                "traffic_note": ("DRAM bytes per launch, scaled from one ncu capture of a "
                                 f"65,536-cell launch ({tb} B/CU)") if tb else
                                "not captured for this kernel",
                "layout": {"bytes_per_cu": bpc, "achieved_gbs": bpc * cu_launch / t_launch / 1e9,
                           "frac": bpc * cu_launch / t_launch / 1e9 / hbm_peak,
                           "note": "bytes this engine's layout streams per CU (cable rows, "
                                   "conductances, CV index, event word; no scratch)"},
                "fp64_pipe": {"achieved": fp64_ach, "peak": fp64_peak, "unit": "TFLOP/s",
                              "frac": fp64_ach / fp64_peak, "fp64_ops_per_cu": fpc,
                              "peak_note": "of measured: pa_measure_fp64 (FP64 FMA chains, CUDA "
                                           "events) x 2 flop, this run",
                              "nominal_tflops": N_SM * DFMA_PER_SM_CLK * 2 * clk * 1e6 / 1e12,
                              "note": "HH divisions count "
                                      f"{RCP64_DFMA_EQ:.2f} FMA-equivalents (measured); the "
                                      "solver's row reciprocal runs on the integer pipes"}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "f32x2 (float-float) solve, sums and conductances + f64 HH and "
                           "plasticity",
                  "fp32": "f64 solve + f32 synapses and mechanisms", "fp64": "f64"}[head],
        "data": "synthetic",
        "config": {"workload": "large_stdp", "n_cells": st["n_cells"], "n_cv": st["n_cv"],
                   "n_synapses": st["n_syn"], "dt_ms": net.dt,
                   "epoch_steps": r["epoch_steps"], "step": "one min-delay epoch",
                   "precision": head, "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": "inputs larger than L2 (working set "
                         f"{r['device_bytes'] / 1e9:.1f} GB vs 126 MB L2)"},
        "roofline": roofline(r, head),
        "gpu_launches": r["kernel_launches"],
        "clocks": r["clocks"],
        "setup_s": r["setup_s"],
    }
    for name, run in runs.items():
        line[name] = {"value": run["n_cv"] * run["epoch_steps"] * args.steps / (run["ms"] * 1e-3),
                      "ms_per_step": run["ms"] / args.steps,
                      "epoch_kernel_ms_per_step": run["epoch_kernel_ms"] / max(run["epoch_launches"], 1),
                      "event_kernels_ms_per_step": run["event_kernels_ms"] / max(run["epoch_launches"], 1),
                      "spikes": run["spikes"], "kernel_shape": run["shape"],
                      "shape_trial_ms": run["shape_trial_ms"],
                      "roofline": roofline(run, name)}
    if "mixed" in runs and "fp64" in runs:
        line["mixed_over_fp64"] = line["mixed"]["value"] / line["fp64"]["value"]
    if "fp32" in runs and "fp64" in runs:
        line["fp32_over_fp64"] = line["fp32"]["value"] / line["fp64"]["value"]
    if not args.no_e2e:
        line["e2e"] = time_e2e(net, precs[head], args.steps, device)
    if not args.no_batched:
        line["batched"] = batched_bench(device)
    if args.serve_jobs > 0:
        line["serving"] = serving_bench(args.serve_jobs, device, alone=not args.serve_no_alone)
    if not args.no_cpu and ws == 1:
        line["cpu_baseline"] = oracle_sample(min(args.cells, 2048), min(args.shapes, 2048))
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
