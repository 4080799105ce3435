"""Pins of the oracle's PRP diffusion (Eq. diffusion on the cell's tree with the
cable solver; synthesis at the soma, degradation everywhere, Eq. prp_single_comp
for the total amount) against closed forms that do not go through the tree
solver: the cosine modes of a uniform chain, the two-compartment exchange, the
single pool's recursion for the total amount, and the limits of very slow and
very fast diffusion."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2411_16445_b300 import workloads as W

H0, THETA_TAG, THETA_PRO, P_MAX, F_INT = 4.20075, 0.840149, 2.10037, 10.0, 0.1


def _cell(morph, d_p, tau_p=100.0, syn_cv=(0,), dt=0.2):
    b = W._Builder(dt, 11, "diff")
    pas = b.mech(W.PAS, W.pas_params())
    stc = b.mech(W.STC, W.stc_params(tau_p=tau_p, d_p=d_p))
    m = b.morph(morph)
    b.cells_add(1, m, pas, pas)
    cv = np.asarray(syn_cv, int)
    b.connect(W.SRC_POISSON, np.zeros(len(cv), int), cv, stc, 1e-3, rate=0.0)
    return b.build()


def _chain(n, length, diam):
    return W.Morphology(parent=np.arange(-1, n - 1, dtype=np.int32),
                        length=np.asarray(np.broadcast_to(length, (n,)), np.float64),
                        diam=np.asarray(np.broadcast_to(diam, (n,)), np.float64),
                        region=np.r_[0, np.ones(n - 1)].astype(np.int32))


def _volumes(m):
    return math.pi * (0.5 * m.diam) ** 2 * m.length


def test_cosine_modes_of_a_uniform_chain():
    """On a uniform chain with closed ends the diffusion operator has the
    eigenvectors cos(pi m (i + 1/2) / n) with rates (2 D / L^2)(1 - cos(pi m / n));
    a backward-Euler step divides mode m by 1 + dt rate, the explicit
    degradation multiplies everything by 1 - dt / tau_p."""
    n, L, D, dt, tau_p, K = 16, 10.0, 10.0, 0.2, 100.0, 200
    net = _cell(_chain(n, L, 2.0), D, tau_p=tau_p, syn_cv=(5,), dt=dt)
    o = O.Oracle(net)
    assert o.has_diffusion(0)
    i = np.arange(n)
    for mode in (1, 3, 15):
        phi = np.cos(math.pi * mode * (i + 0.5) / n)
        o.set_prp(1.0 + 0.5 * phi)
        k0 = o.step_count()
        o.run(K)
        assert o.step_count() == k0 + K
        lam = (2 * D / L ** 2) * (1 - math.cos(math.pi * mode / n))
        r = dt / tau_p
        want = (1 - r) ** K + 0.5 * ((1 - r) / (1 + dt * lam)) ** K * phi
        assert np.allclose(o.prp(), want, rtol=0, atol=1e-12)
        assert o.cell_p()[0] == o.prp()[0]


def test_two_compartment_exchange():
    """Two cylinders of different radii: the amount sum V_i P_i only degrades;
    the difference P_1 - P_0 relaxes at g (1/V_0 + 1/V_1), g the conductance of
    two half-cylinders in series (diffusive resistance (L/2) / (D pi r^2) each)."""
    m = W.Morphology(parent=np.array([-1, 0], np.int32), length=np.array([10.0, 20.0]),
                     diam=np.array([10.0, 2.0]), region=np.array([0, 1], np.int32))
    D, dt, tau_p, K = 2.0, 0.2, 1000.0, 300
    o = O.Oracle(_cell(m, D, tau_p=tau_p, dt=dt))
    o.set_prp(np.array([1.0, 0.0]))
    o.run(K)
    V = _volumes(m)
    R = (0.5 * m.length) / (D * math.pi * (0.5 * m.diam) ** 2)
    g = 1.0 / R.sum()
    r = dt / tau_p
    P = o.prp()
    assert math.isclose(V @ P, V[0] * (1 - r) ** K, rel_tol=1e-12)
    want = -((1 - r) / (1 + dt * g * (1 / V[0] + 1 / V[1]))) ** K
    assert math.isclose(P[1] - P[0], want, rel_tol=1e-11)


@pytest.mark.parametrize("seed", [1, 2])
def test_total_amount_follows_the_single_pool(seed):
    """Summed over the tree, synthesis p_max V_tot / tau_p at the soma and
    degradation P / tau_p in every CV give the single pool's forward-Euler
    recursion for the mean concentration: A' = (1 - r) A + r q V_tot, with q =
    p_max while the summed early-phase change S exceeds theta_pro."""
    rng = np.random.default_rng(seed)
    morph = W.random_binary_tree(rng, 12)
    n = morph.n_cv
    syn_cv = rng.integers(0, n, 30)
    dt, tau_p = 0.2, 40.0
    net = _cell(morph, 0.5, tau_p=tau_p, syn_cv=syn_cv, dt=dt)
    o = O.Oracle(net)
    # tags above theta_pro for a while, then h = h0 (no synthesis)
    o.set_syn(O.SYN_H, H0 + rng.uniform(0.05, 0.2, net.n_conn))
    V = _volumes(morph)
    vtot = V.sum()
    r = dt / tau_p
    A = 0.0
    seen = set()
    for k in range(400):
        if k == 250:
            o.set_syn(O.SYN_H, np.full(net.n_conn, H0))
        S = np.abs(o.syn(O.SYN_H) - H0).sum()
        q = P_MAX if S > THETA_PRO else 0.0
        seen.add(q)
        A = (1 - r) * A + r * q * vtot
        o.run(1)
        assert math.isclose(V @ o.prp(), A, rel_tol=1e-12, abs_tol=1e-300)
    assert seen == {0.0, P_MAX}
    assert np.all(o.prp() >= 0)


def test_z_captures_the_local_prp():
    """Eq. late_phase_weight with the PRP at the synapse's own CV."""
    rng = np.random.default_rng(5)
    morph = _chain(8, 10.0, 2.0)
    syn_cv = np.array([0, 3, 7, 7])
    dt = 0.2
    net = _cell(morph, 1.0, syn_cv=syn_cv, dt=dt)
    o = O.Oracle(net)
    P = rng.uniform(0.5, 5.0, 8)
    o.set_prp(P)
    o.set_syn(O.SYN_H, np.array([H0 + 1.0, H0 + 2.0, H0 - 1.0, H0]))
    o.run(1)
    rz = dt / 3600.0e3
    want = rz * np.array([P[0] * F_INT, P[3] * F_INT, -(P[7] * F_INT) * 0.5, 0.0])
    assert np.allclose(o.syn(O.SYN_Z), want, rtol=1e-15, atol=0)


def test_slow_and_fast_diffusion_limits():
    """D -> 0: the synthesised PRP stays in the soma CV; D -> infinity: the field
    is uniform at the single pool's concentration."""
    morph = _chain(10, 10.0, 2.0)
    dt, tau_p, K = 0.2, 50.0, 100
    r = dt / tau_p
    mean = P_MAX * (1 - (1 - r) ** K)
    V = _volumes(morph)
    for D, check in ((1e-9, "soma"), (1e6, "uniform")):
        net = _cell(morph, D, tau_p=tau_p, syn_cv=(4,), dt=dt)
        o = O.Oracle(net)
        o.set_syn(O.SYN_H, np.full(1, H0 + 3.0))
        o.run(K)
        P = o.prp()
        assert math.isclose(V @ P, mean * V.sum(), rel_tol=1e-11)
        if check == "soma":
            assert math.isclose(P[0], mean * V.sum() / V[0], rel_tol=1e-6)
            assert np.all(P[1:] < 1e-6 * P[0])
        else:
            assert np.allclose(P, mean, rtol=1e-3)


def test_single_cv_matches_the_single_pool():
    """A one-CV cell: diffusion changes nothing, the field is the cell's pool."""
    nets = [_cell(W.soma_only(20.0), d, tau_p=30.0, syn_cv=(0, 0), dt=0.1) for d in (0.0, 3.0)]
    oo = [O.Oracle(n) for n in nets]
    assert not oo[0].has_diffusion(0) and oo[1].has_diffusion(0)
    for o in oo:
        o.set_syn(O.SYN_H, np.array([H0 + 2.0, H0 + 1.5]))
    for _ in range(5):
        for o in oo:
            o.run(200)
        assert math.isclose(oo[0].cell_p()[0], oo[1].cell_p()[0], rel_tol=1e-13)
        assert oo[1].prp()[0] == oo[1].cell_p()[0]
        assert np.allclose(oo[0].syn(O.SYN_Z), oo[1].syn(O.SYN_Z), rtol=1e-12)


def test_fast_forward_long_steps_of_the_field():
    """Fast-forward: the field takes backward-Euler diffusion steps of the long
    step (chain modes divided by 1 + dtl rate) and the explicit degradation of
    the long step; the amount follows the single pool's long-step recursion."""
    n, L, D, dt, tau_p = 16, 10.0, 10.0, 0.2, 5000.0
    o = O.Oracle(_cell(_chain(n, L, 2.0), D, tau_p=tau_p, syn_cv=(5,), dt=dt))
    i = np.arange(n)
    phi = np.cos(math.pi * 2 * (i + 0.5) / n)
    o.set_prp(1.0 + 0.5 * phi)
    K, n_long = 50_000, 40                          # 10 s in 40 steps of 250 ms
    o.fast_forward(K, n_long)
    dtl = K * dt / n_long
    lam = (2 * D / L ** 2) * (1 - math.cos(math.pi * 2 / n))
    r = dtl / tau_p
    want = (1 - r) ** n_long + 0.5 * ((1 - r) / (1 + dtl * lam)) ** n_long * phi
    assert np.allclose(o.prp(), want, rtol=0, atol=1e-12)
    # with synthesis: the amount follows A' = (1 - r) A + r p_max V_tot
    rng = np.random.default_rng(4)
    morph = W.random_binary_tree(rng, 10)
    o = O.Oracle(_cell(morph, 0.3, tau_p=tau_p, syn_cv=rng.integers(0, morph.n_cv, 12), dt=dt))
    o.set_syn(O.SYN_H, np.full(12, H0 + 1.0))      # S = 12 > theta_pro, tagged, constant
    o.fast_forward(K, n_long)
    V = _volumes(morph)
    A = 0.0
    for _ in range(n_long):
        A = (1 - r) * A + r * P_MAX * V.sum()
    assert math.isclose(V @ o.prp(), A, rel_tol=1e-12)
    assert o.step_count() == K


def test_bad_diffusivity():
    net = _cell(_chain(4, 10.0, 2.0), 1.0)
    net.mech_params[1][-1] = -1.0
    with pytest.raises(ValueError):
        O.Oracle(net)
