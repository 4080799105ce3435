"""Pins of the oracle's plasticity noise (Eqs. plasticity_noise_1-2; Sec.
"Computation with stochastic differential equations"): the model's logarithm
and circular functions against the C library, the Box-Muller deviates against
an independent recomputation from the Threefry words, their statistics, and
the Euler-Maruyama variance of the weight when the calcium stays above both
thresholds."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_2411_16445_b300 import workloads as W


def test_model_log_within_two_ulp_of_libm():
    rng = np.random.default_rng(11)
    xs = np.concatenate([rng.random(20000), np.exp(-rng.random(5000) * 700.0),
                         np.exp(rng.random(5000) * 700.0), [1.0, 0.5, 2.0 ** -53, 1 - 2.0 ** -53]])
    for x in xs:
        ref = math.log(x)
        assert abs(O.log(x) - ref) <= 2 * math.ulp(ref) + 1e-300, x


def test_model_sin_cos_of_two_pi_v():
    rng = np.random.default_rng(12)
    vs = np.concatenate([rng.random(20000), [0.0, 0.125, 0.25, 0.375, 0.5, 0.625, 0.75, 0.875,
                                             1 - 2.0 ** -53]])
    for v in vs:
        assert abs(O.cis2pi(v, 0) - math.cos(2 * math.pi * v)) <= 1e-15
        assert abs(O.cis2pi(v, 1) - math.sin(2 * math.pi * v)) <= 1e-15
    assert O.cis2pi(0.0, 0) == 1.0 and O.cis2pi(0.0, 1) == 0.0


def test_normal_is_box_muller_of_the_threefry_words():
    """Counter (id, step/4, 2, 0), key (seed, 0, 0, 0); step mod 4 = 2p + j uses
    words 2p, 2p+1 as 53-bit uniforms; cos for j = 0, sin for j = 1."""
    seed = 0x5EED5EED12345
    for noise_id in (0, 7, 123456):
        for step in range(0, 40):
            w = O.threefry([noise_id, step >> 2, 2, 0], [seed, 0, 0, 0])
            j = step & 3
            u1 = int(w[j & 2] >> np.uint64(11)) * 2.0 ** -53
            u2 = int(w[(j & 2) + 1] >> np.uint64(11)) * 2.0 ** -53
            ang = 2 * math.pi * u2
            ref = math.sqrt(-2 * math.log(1 - u1)) * (math.sin(ang) if j & 1 else math.cos(ang))
            assert abs(O.normal(seed, noise_id, step) - ref) <= 1e-13 * max(1.0, abs(ref))


def test_normal_statistics():
    z = np.array([O.normal(20241125, i, k) for i in range(400) for k in range(250)])
    assert abs(z.mean()) < 0.015 and abs(z.var() - 1.0) < 0.02
    assert stats.kstest(z, "norm").pvalue > 1e-3
    zz = z.reshape(400, 250)
    lag = np.mean(zz[:, 1:] * zz[:, :-1])
    assert abs(lag) < 0.015                      # consecutive steps of one source
    assert abs(np.mean(zz[1:] * zz[:-1])) < 0.015  # neighbouring sources


def _held_calcium_net(kind, n_syn, sigma, c_pre, dt=0.025):
    """One passive cell with n_syn GB or STC synapses, each driven by its own
    10 kHz Poisson train, calcium jumps of c_pre with tau_c = 1e12 ms (held),
    no delay, no potentiation or depression terms."""
    b = W._Builder(dt, 99, "noise")
    pas = b.mech(W.PAS, W.pas_params())
    if kind == "gb":
        syn = b.mech(W.GB, W.gb_params(tau_c=1e12, c_pre=c_pre, c_post=0.0, gamma_p=0.0,
                                       gamma_d=0.0, w0=0.5, w_star=0.5, t_c_delay=0.0,
                                       sigma_pl=sigma))
    else:
        syn = b.mech(W.STC, W.stc_params(tau_c=1e12, c_pre=c_pre, c_post=0.0, gamma_p=0.0,
                                         gamma_d=0.0, t_c_delay=0.0, sigma_pl=sigma))
    m = b.morph(W.soma_only(20.0))
    b.cells_add(1, m, pas, pas)
    b.connect(W.SRC_POISSON, np.zeros(n_syn, int), 0, syn, 0.0, rate=10000.0)
    return b.build()


@pytest.mark.parametrize("kind,field,tau,sigma,x0", [
    ("gb", O.SYN_W, 346.0e3, 2.8248, 0.5),        # Table 3
    ("stc", O.SYN_H, 688.4e3, 2.90436, 4.20075),  # Table 5
])
def test_euler_maruyama_variance_with_calcium_above_both_thresholds(kind, field, tau, sigma, x0):
    """Calcium above theta_p and theta_d from each synapse's first event on: the
    weight takes sigma sqrt(2 dt / tau) N(0,1) per step (the drift at the start
    value is zero or negligible over 4000 steps), so after n steps its variance
    over synapses is n sigma^2 2 dt / tau."""
    n_syn, steps, dt = 1500, 4000, 0.025
    o = O.Oracle(_held_calcium_net(kind, n_syn, sigma, c_pre=1e6, dt=dt))
    o.run(steps)
    x = o.syn(field)
    assert np.all(o.syn(O.SYN_C) > 1e5)
    want = steps * sigma ** 2 * 2 * dt / tau       # the few steps before the first event aside
    assert abs(x.var() / want - 1.0) < 0.15
    assert abs(x.mean() - x0) < 4 * math.sqrt(want / n_syn)


@pytest.mark.parametrize("kind,field", [("gb", O.SYN_W), ("stc", O.SYN_H)])
def test_noise_gated_by_the_thresholds_and_off_at_zero_sigma(kind, field):
    """Calcium below both thresholds: no noise at all (bit-identical to sigma = 0);
    and sigma = 0 with the calcium above them is the deterministic rule."""
    quiet = [O.Oracle(_held_calcium_net(kind, 50, s, c_pre=1e-3)) for s in (0.0, 3.0)]
    for o in quiet:
        o.run(2000)
    assert np.array_equal(quiet[0].syn(field), quiet[1].syn(field))
    loud = [O.Oracle(_held_calcium_net(kind, 50, s, c_pre=1e6)) for s in (0.0, 3.0)]
    for o in loud:
        o.run(2000)
    assert not np.array_equal(loud[0].syn(field), loud[1].syn(field))
