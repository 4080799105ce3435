"""Pins of the oracle's fast-forward (the '8h-recall' paradigm: long biological
times without spiking and calcium dynamics, the slow plasticity variables in
long forward-Euler steps) against the closed forms of that scheme."""
import math

import numpy as np
from scipy.integrate import solve_ivp

import oracle as O
from paper_2411_16445_b300 import workloads as W


def _stc_cell(n_syn=40, dt=0.2):
    b = W._Builder(dt, 7, "ff")
    pas = b.mech(W.PAS, W.pas_params())
    stc = b.mech(W.STC, W.stc_params())
    m = b.morph(W.soma_only(20.0))
    b.cells_add(1, m, pas, pas)
    b.connect(W.SRC_POISSON, np.zeros(n_syn, int), 0, stc, 1e-3, rate=0.0)
    return b.build()


def test_h_relaxes_and_z_stays_without_prp():
    net = _stc_cell()
    o = O.Oracle(net)
    h0 = 4.20075
    d = np.random.default_rng(1).uniform(-0.5, 0.5, net.n_conn)
    o.set_syn(O.SYN_H, h0 + d)
    K, n = 50000, 20                                   # 10 s in 20 long steps of 500 ms
    o.fast_forward(K, n)
    r = (K * net.dt / n) / 688.4e3
    assert np.allclose(o.syn(O.SYN_H) - h0, d * (1 - 0.1 * r) ** n, rtol=1e-9, atol=1e-14)
    assert np.all(o.syn(O.SYN_Z) == 0.0) and o.step_count() == K


def test_prp_saturates_and_tagged_z_follows_its_closed_form():
    net = _stc_cell(n_syn=40)
    o = O.Oracle(net)
    h0, theta_tag, f_int, p_max = 4.20075, 0.840149, 0.1, 10.0
    o.set_syn(O.SYN_H, np.full(net.n_conn, h0 + 3.0))  # S = 40 x 3 >> theta_pro; all tagged
    K, n = 180000, 36                                   # 1 h in 100 s steps
    dtl = K * net.dt / n
    o.fast_forward(K, n)
    # p from 0: p_max (1 - (1 - dtl / tau_p)^n)
    rp = dtl / 3600.0e3
    assert math.isclose(o.cell_p()[0], p_max * (1 - (1 - rp) ** n), rel_tol=1e-12)
    # the z recursion with the p sequence above (z uses the cell's p before its update)
    rz = dtl / 3600.0e3
    z, p = 0.0, 0.0
    for _ in range(n):
        z = z + rz * (p * f_int * (1 - z))
        p = p + rp * (p_max - p)
    assert np.allclose(o.syn(O.SYN_Z), z, rtol=1e-12)
    assert np.all(o.syn(O.SYN_H) - h0 > theta_tag)      # still tagged throughout


def test_gb_weight_drift_fixed_points_and_ode_limit():
    dt = 0.1
    b = W._Builder(dt, 3, "ffgb")
    pas = b.mech(W.PAS, W.pas_params())
    gb = b.mech(W.GB, W.gb_params(w_star=0.5))
    m = b.morph(W.soma_only(20.0))
    b.cells_add(1, m, pas, pas)
    b.connect(W.SRC_POISSON, np.zeros(5, int), 0, gb, 1e-3, rate=0.0)
    o = O.Oracle(b.build())
    w0 = np.array([0.0, 0.5, 1.0, 0.3, 0.7])
    o.set_syn(O.SYN_W, w0)
    K, n = 10_000_000, 2000                          # 1000 s in 0.5 s steps
    o.fast_forward(K, n)
    w = o.syn(O.SYN_W)
    assert w[0] == 0.0 and w[1] == 0.5 and w[2] == 1.0  # fixed points of the cubic
    tau = 346.0e3
    for x0, x in zip(w0[3:], w[3:]):
        sol = solve_ivp(lambda t, y: -(y * (1 - y) * (0.5 - y)) / tau, (0, K * dt), [x0],
                        rtol=1e-12, atol=1e-14)
        assert abs(x - sol.y[0, -1]) < 5e-4 * abs(x0 - 0.5)  # first order in the long step
        assert (x - 0.5) * (x0 - 0.5) > 0 and abs(x - 0.5) > abs(x0 - 0.5)


def test_decay_and_clock():
    """g and c decay by exactly exp(-K dt / tau) and the clock moves on by K."""
    net = W.single_neuron()
    o = O.Oracle(net)
    o.run(4000)
    g, c = o.syn(O.SYN_G), o.syn(O.SYN_C)
    K = 3
    o.fast_forward(K, 1)
    T = K * net.dt
    assert np.array_equal(o.syn(O.SYN_G), g * np.exp(-T / 5.0))
    assert np.array_equal(o.syn(O.SYN_C), c * np.exp(-T / 20.0))
    assert o.step_count() == 4000 + K
