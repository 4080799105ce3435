"""Continuous-batching server: a job's results are the same alone and among other
jobs (same precision: bit-identical, since jobs share no device state and a
batch member takes exactly its own steps), budget admission never exceeds the
budget estimate, and latency is reported."""
import numpy as np
import pytest

from paper_2411_16445_b300 import workloads as W
from paper_2411_16445_b300 import serving as S


def small_trace(n=12, seed=5):
    return W.serving_trace(n_jobs=n, rate_hz=40.0, seed=seed, sizes=(1, 300),
                           durations_s=(0.02, 0.2))


def test_trace_statistics_and_estimates():
    tr = W.serving_trace(n_jobs=400, rate_hz=20.0, seed=3)
    arr = np.array([j["arrival_s"] for j in tr])
    assert np.all(np.diff(arr) > 0)
    rate = (len(arr) - 1) / (arr[-1] - arr[0])
    assert 16.0 < rate < 24.0
    n = np.array([j["n_cells"] for j in tr])
    assert n.min() >= 1 and n.max() <= 20000
    # log-uniform: about half the jobs below the geometric midpoint (~141 cells)
    assert 0.4 < np.mean(n < np.sqrt(20000)) < 0.6
    for j in tr[:20]:
        if j["n_cells"] > 3000:
            continue
        net = W.serving_job(j["n_cells"], j["long_dendrite"], j["dend_len_um"],
                            j["dend_diam_um"], j["seed"], dt=j["dt"])
        assert S.estimate_spec_bytes(j) >= 0.95 * S.estimate_bytes(net)


@pytest.mark.gpu
def test_results_alone_equal_results_in_the_mix():
    from paper_2411_16445_b300 import engine as E
    trace = small_trace()
    srv = S.Server(hbm_budget_bytes=2 << 30, epochs_per_tick=2, precision=E.PA_MIXED)
    out = srv.run(trace)
    assert len(out["results"]) == len(trace)
    assert out["p50_s"] is not None and out["p99_s"] >= out["p50_s"] > 0
    assert out["graph_launches"] > 0      # the jobs did run as one batch
    for r, spec in zip(out["results"], sorted(trace, key=lambda j: j["job_id"])):
        n_cv, steps, g, s, w = S.run_alone(spec, precision=E.PA_MIXED)
        assert r.steps == steps and r.n_cv == n_cv
        assert r.spikes == len(g) and r.spike_digest == S.spike_digest(g, s)
        assert np.array_equal(r.weights, w)


@pytest.mark.gpu
def test_budget_limits_residency():
    from paper_2411_16445_b300 import engine as E
    trace = small_trace(8, seed=9)
    biggest = max(S.estimate_spec_bytes(j) for j in trace)
    # a budget for one job at a time still completes every job, one after another
    srv = S.Server(hbm_budget_bytes=biggest, epochs_per_tick=8, precision=E.PA_MIXED)
    out = srv.run(trace)
    assert len(out["results"]) == len(trace)
    starts = sorted((r.start_s, r.done_s) for r in out["results"])
    for (s0, d0), (s1, d1) in zip(starts, starts[1:]):
        assert s1 >= d0 - 1e-3  # never two resident jobs at once
