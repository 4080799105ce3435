"""Pins of the oracle's heterosynaptic calcium rule (Eqs.
ca_injection_current_spine, ca_diffusion_dendrite, heterosyn_weight) against
closed forms: the injection current's exponential decay after a jump of I0,
the calcium of one isolated CV under that inflow, the forward-Euler weight
rule in each calcium regime, the total amount under diffusion, and the
chain's cosine modes."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2411_16445_b300 import workloads as W

F = 96485.33212


def _cell(morph, syn_cv, params, dt=0.025, seed=3):
    """one cell with HCA synapses on syn_cv, driven by a replayed source cell"""
    b = W._Builder(dt, seed, "hca")
    pas = b.mech(W.PAS, W.pas_params())
    h = b.mech(W.HCA, W.hca_params(**params))
    m = b.morph(morph)
    src = b.morph(W.soma_only(10.0))
    b.cells_add(1, m, pas, pas)
    b.cells_add(1, src, pas, pas)
    cv = np.asarray(syn_cv)
    b.connect(1, np.zeros(len(cv), int), cv, h, 1.0, delay=dt)
    return b.build()


def _chain(n, length=1.0, diam=2.0):
    return W.Morphology(np.arange(-1, n - 1, dtype=np.int32), np.full(n, length),
                        np.full(n, diam), np.r_[0, np.ones(n - 1)].astype(np.int32))


def test_single_cv_current_and_calcium():
    """One isolated CV, one synapse, one event: I = I0 e^{-(k - k_e) dt / tau_I}
    after the jump; C follows C' = C + r (q - C), q = tau_C w gamma I / (2 F V);
    no plasticity (thresholds out of reach)."""
    dt, i0, tau_i, gamma, tau_c, w0 = 0.025, 4.0, 1.0, 0.11, 100.0, 0.5
    p = dict(i0=i0, tau_i=tau_i, gamma=gamma, theta_p=1e9, theta_d=1e9, w0=w0, tau_c=tau_c, d=0.3)
    net = _cell(W.soma_only(8.0), [0], p, dt=dt)
    o = O.Oracle(net)
    k_spike = 40
    o.set_replay(np.array([1], np.int32), np.array([k_spike], np.int64))
    V = math.pi * 4.0 ** 2 * 8.0
    kq = gamma * 1e6 / (2 * F)
    r = dt / tau_c
    C, I = 0.0, 0.0
    decay = math.exp(-dt / tau_i)
    for k in range(400):
        if k == k_spike + 1:                 # delivered one step (the delay) later
            I += i0
        q = tau_c * (w0 * (kq * I)) / V
        C = C + r * (q - C)
        I *= decay
        o.run(1)
        assert math.isclose(o.syn(O.SYN_C)[0], I, rel_tol=1e-12, abs_tol=1e-300)
        assert math.isclose(o.ca()[0], C, rel_tol=1e-11, abs_tol=1e-300)
    assert o.syn(O.SYN_W)[0] == w0
    assert C > 0.0


@pytest.mark.parametrize("level,regime", [(0.2, "both"), (0.08, "depression"), (0.01, "none")])
def test_weight_rule_in_each_regime(level, regime):
    """Eq. heterosyn_weight, forward Euler with the calcium of the synapse's CV
    before the step's update: potentiation (1 - w) gamma_p above theta_p,
    depression w gamma_d above theta_d (rates per second)."""
    dt, gp, gd, thp, thd = 0.025, 90.0, 0.01, 0.11, 0.05
    p = dict(gamma_p=gp, gamma_d=gd, theta_p=thp, theta_d=thd, w0=0.3)
    net = _cell(_chain(3), [1], p, dt=dt)
    o = O.Oracle(net)
    w = 0.3
    for _ in range(200):
        c = np.full(o.ca().shape, level)
        o.set_ca(c)
        Pp = (dt * gp * 1e-3) * (1 - w) if level > thp else 0.0
        Dd = (dt * gd * 1e-3) * w if level > thd else 0.0
        w = w + (Pp - Dd)
        o.run(1)
        assert o.syn(O.SYN_W)[0] == pytest.approx(w, rel=1e-14, abs=0)
    if regime == "both":
        w_star = gp / (gp + gd)
        assert abs(w - w_star) < abs(0.3 - w_star)
    elif regime == "depression":
        assert w < 0.3
    else:
        assert w == 0.3


def test_amount_under_diffusion():
    """On a tree with diffusion, sum V_i C_i follows A' = (1 - r) A + dt S_k,
    S_k = sum over synapses of w gamma I_k / (2 F): the diffusion conserves,
    the decay is the explicit reaction's."""
    rng = np.random.default_rng(8)
    morph = W.random_binary_tree(rng, 20)
    cvs = [0, 5, 5, 11]
    dt, tau_c = 0.025, 50.0
    p = dict(theta_p=1e9, theta_d=1e9, tau_c=tau_c, d=0.5, tau_i=2.0)
    net = _cell(morph, cvs, p, dt=dt)
    o = O.Oracle(net)
    o.set_replay(np.ones(6, np.int32), np.array([10, 20, 30, 60, 61, 90], np.int64))
    V = math.pi * (0.5 * morph.diam) ** 2 * morph.length
    kq = 0.11 * 1e6 / (2 * F)
    r = dt / tau_c
    A = 0.0
    for k in range(300):
        I = o.syn(O.SYN_C)                      # after the previous step's decay
        # this step's events jump I before its use
        ev = (k - 1) in (10, 20, 30, 60, 61, 90)
        I_use = I + (4.0 if ev else 0.0)
        S = float(np.sum(0.5 * (kq * I_use)))
        A = (1 - r) * A + dt * S
        o.run(1)
        n = morph.n_cv
        assert math.isclose(V @ o.ca()[:n], A, rel_tol=1e-11, abs_tol=1e-300)
    assert A > 0


def test_chain_cosine_modes_without_input():
    """Without inflow the field decays by (1 - r) per step and mode m of a
    uniform chain is divided by 1 + dt (2 D / L^2)(1 - cos(pi m / n))."""
    n, D, dt, tau_c, K = 20, 0.22, 0.025, 100.0, 400
    net = _cell(_chain(n), [3], dict(d=D, tau_c=tau_c), dt=dt)
    o = O.Oracle(net)
    i = np.arange(n)
    mode = 2
    phi = np.cos(math.pi * mode * (i + 0.5) / n)
    c0 = np.zeros(o.ca().shape)
    c0[:n] = 0.1 + 0.05 * phi
    o.set_ca(c0)
    o.run(K)
    lam = (2 * D / 1.0 ** 2) * (1 - math.cos(math.pi * mode / n))
    r = dt / tau_c
    want = 0.1 * (1 - r) ** K + 0.05 * ((1 - r) / (1 + dt * lam)) ** K * phi
    assert np.allclose(o.ca()[:n], want, rtol=0, atol=1e-13)


def test_no_conductance_and_fast_forward_refused():
    net, (gid, step) = W.heterosyn_dendrite(n_spikes=3)
    o = O.Oracle(net)
    o.set_replay(gid, step)
    o.run(800)
    assert np.all(o.syn(O.SYN_G) == 0.0)        # the calcium current is not electrical
    assert np.all(np.abs(o.v() - (-65.0)) < 12.0)
    ca = o.ca()
    assert ca[80] > 0 and ca[82] > 0            # the active heads
    with pytest.raises(ValueError):
        O.Oracle(net).fast_forward(100, 2)
