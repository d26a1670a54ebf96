"""Pins of the oracle parts of the current-based cortex variant: the BC2008
model table against the published rate formulas written out directly, the
background normal's moments and histogram, the compound Poisson x Gaussian
background's mean and variance against the closed forms of a compound
Poisson sum, and current-based synaptic delivery against the same neuron
given the post-synaptic current waveform explicitly."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2601_21407_gb300 import inputs as inp


def _bc(VT):
    """Pospischil et al. 2008: the Traub-Miles rates with threshold V_T and
    the M current, in their printed form (1/ms, mV)."""
    return {
        "am": lambda V: -0.32 * (V - VT - 13) / (math.exp(-(V - VT - 13) / 4) - 1),
        "bm": lambda V: 0.28 * (V - VT - 40) / (math.exp((V - VT - 40) / 5) - 1),
        "ah": lambda V: 0.128 * math.exp(-(V - VT - 17) / 18),
        "bh": lambda V: 4 / (1 + math.exp(-(V - VT - 40) / 5)),
        "an": lambda V: -0.032 * (V - VT - 15) / (math.exp(-(V - VT - 15) / 5) - 1),
        "bn": lambda V: 0.5 * math.exp(-(V - VT - 10) / 40),
        "pinf": lambda V: 1 / (1 + math.exp(-(V + 35) / 10)),
        "taup": lambda V, tmax: tmax / (3.3 * math.exp((V + 35) / 20) + math.exp(-(V + 35) / 20)),
    }


@pytest.mark.parametrize("model,VT,tmax", [(inp.BC2008_RS, -56.2, 608.0), (inp.BC2008_FS, -57.9, 502.0)])
def test_bc2008_table_is_the_published_model(model, VT, tmax):
    ref = _bc(VT)
    g = [gt for ch in model["channels"] for gt in ch["gates"]]
    for V in np.linspace(-95.0, 40.0, 271) + 0.0137:  # off the removable points
        got = [oracle.rate(g[0]["f1"], V), oracle.rate(g[0]["f2"], V), oracle.rate(g[1]["f1"], V),
               oracle.rate(g[1]["f2"], V), oracle.rate(g[2]["f1"], V), oracle.rate(g[2]["f2"], V),
               oracle.rate(g[3]["f1"], V), oracle.rate(g[3]["f2"], V)]
        want = [ref["am"](V), ref["bm"](V), ref["ah"](V), ref["bh"](V), ref["an"](V), ref["bn"](V),
                ref["pinf"](V), ref["taup"](V, tmax)]
        assert np.allclose(got, want, rtol=1e-9, atol=0), (V, got, want)
    E = {ch["name"]: ch["E"] for ch in model["channels"]}
    assert E["Na"] == 50.0 and E["Kd"] == -90.0 and E["M"] == -90.0


def test_background_normal_moments():
    z = np.array([oracle.background_normal(7, t, i) for t in range(400) for i in range(500)])
    n = z.size
    assert abs(z.mean()) < 4 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 4 * math.sqrt(2.0 / n)
    edges = np.array([-np.inf, -2, -1.5, -1, -0.5, 0, 0.5, 1, 1.5, 2, np.inf])
    obs = np.histogram(z, edges)[0]
    exp = n * np.diff(stats.norm.cdf(edges))
    assert stats.chisquare(obs, exp).pvalue > 1e-3


def test_compound_background_moments():
    """k ~ Poisson(lambda), amplitude ~ N(k mu, k sigma^2): mean lambda mu,
    variance lambda (mu^2 + sigma^2) (a compound Poisson sum); the
    fixed-weight form (sigma = 0) gives variance lambda mu^2."""
    K, rate, dt, mu, sd = 2000, 8.0, 0.1, 0.17, 0.017
    lam = K * rate * dt / 1000.0
    x = np.array([oracle.background_input(3, t, i, K, rate, dt, mu, sd) for t in range(300) for i in range(400)])
    n = x.size
    var = lam * (mu * mu + sd * sd)
    assert abs(x.mean() - lam * mu) < 4 * math.sqrt(var / n)
    assert abs(x.var() - var) / var < 0.03
    y = np.array([oracle.background_input(3, t, i, K, rate, dt, mu, 0.0) for t in range(300) for i in range(400)])
    assert abs(y.var() - lam * mu * mu) / (lam * mu * mu) < 0.03
    # the same counts: the two differ only where k > 0, by sqrt(k) sd z
    assert np.array_equal(x == 0, y == 0)


def test_current_synapse_delivery():
    """Open loop with current-based synapses: neuron 2 gets an excitatory
    synapse (weight 0.9) from neuron 0 and an inhibitory one (1.3) from
    neuron 1; forced spikes at steps 5 and 30 arrive D steps later and decay
    with tau_E / tau_I.  Neuron 2's trace equals the point neuron given
    I(t) = 0.9 dE^(t - 5 - D) - 1.3 dI^(t - 30 - D) (from the arrivals on)."""
    dt, D, T = 0.1, 15, 400
    syn = {"tau_E": 0.5, "tau_I": 0.5, "E_E": 0.0, "E_I": -80.0, "area_cm2": 2e-4}
    net = {"row_ptr": np.array([0, 0, 0, 2], np.int64), "col": np.array([0, 1], np.int32),
           "w": np.array([0.9, 1.3]), "inh": np.array([0, 1, 0], np.uint8),
           "V0": np.array([-70.0, -70.0, -70.0])}
    forced = (np.array([5, 30], np.int32), np.array([0, 1], np.int32))
    r = oracle.simulate_network(inp.BC2008_RS, net, T, dt, D, syn, forced=forced, syn_current=True,
                                trace_idx=np.array([2]))
    t = np.arange(T)
    dE = math.exp(-dt / syn["tau_E"])
    I = np.where(t >= 5 + D, 0.9 * dE ** (t - 5 - D), 0.0) - np.where(t >= 30 + D, 1.3 * dE ** (t - 30 - D), 0.0)
    ref = oracle.simulate(inp.BC2008_RS, [0.0], [-70.0], T, dt, I_steps=I[:, None])
    assert np.abs(r["V"][:, 0] - ref["V"][:, 0]).max() < 1e-10
    assert r["V"][:5 + D, 0].max() - r["V"][0, 0] < 1e-3 < r["V"][5 + D + 3, 0] - r["V"][5 + D, 0]
