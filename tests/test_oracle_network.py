"""Pins of the FP64 oracle's network path: Philox known answers, the Poisson
sampler, routing against dense brute force, the delay line, a pure-Python
brute-force network, and a passive membrane against an ODE solver (CPU)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2601_21407_gb300 import inputs as inp

HH = inp.CLASSIC_HH
GOLD = os.path.join(os.path.dirname(__file__), "golden")
SYN = {"tau_E": 5.0, "tau_I": 10.0, "E_E": 0.0, "E_I": -80.0, "area_cm2": 2.0e-4}
PASSIVE = {"name": "passive", "C_m": 1.0, "calcium": None,
           "channels": [{"name": "L", "E": -65.0, "gbar": 0.1, "gates": []}]}


def test_philox_known_answers():
    with open(os.path.join(GOLD, "philox4x32_10_kat.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox4x32_10(v[0:4], v[4:6]) == v[6:10]


@pytest.mark.parametrize("lam", [0.0263, 0.263, 2.5, 12.0])
def test_poisson_table_against_scipy(lam):
    """thr[j] = floor(2^32 F(j)) with F the Poisson CDF; scipy's CDF agrees to
    a couple of units of 2^-32 (different summation)."""
    st = pytest.importorskip("scipy.stats")
    thr = oracle.poisson_table(lam)
    assert thr[-1] == 1 << 32
    ref = np.floor(st.poisson.cdf(np.arange(thr.size), lam) * 2.0**32)
    ok = thr[:-1].astype(np.float64)
    assert np.all(np.abs(ok - ref[:-1]) <= 2.0)
    assert np.all(np.diff(thr.astype(np.float64)) >= 0)


def test_poisson_sampler_moments():
    """Counts drawn by the background mapping (Philox word -> inverse CDF)
    have mean and variance lambda within 4 sigma over 1e6 draws, and the
    count frequencies follow the pmf (chi-square)."""
    st = pytest.importorskip("scipy.stats")
    lam = oracle.background_lambda(2106, 5.0, 0.025)
    assert lam == pytest.approx(0.26325, rel=1e-12)
    thr = oracle.poisson_table(lam)
    n = 1_000_000
    ks = np.array([oracle.poisson_sample(oracle.background_word(7, t, i), thr)
                   for t in range(100) for i in range(n // 100)])
    m, v = ks.mean(), ks.var()
    assert abs(m - lam) < 4 * math.sqrt(lam / n)
    # var of the sample variance ~ (mu4 - sigma^4)/n, mu4 = lam(1+3 lam)
    assert abs(v - lam) < 4 * math.sqrt((lam * (1 + 3 * lam) - lam**2) / n)
    obs = np.bincount(ks, minlength=6)[:5].astype(float)
    exp = st.poisson.pmf(np.arange(5), lam) * n
    chi2 = ((obs - exp) ** 2 / exp).sum()
    assert chi2 < st.chi2.ppf(0.9999, 4)


def _dense(n, row_ptr, col, w):
    W = np.zeros((n, n))
    for i in range(n):
        for e in range(row_ptr[i], row_ptr[i + 1]):
            W[i, col[e]] += w[e]
    return W


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_routing_matches_dense_brute_force(seed):
    """CSR push routing == dense matrix-vector brute force, bit for bit in
    2^-32 nS fixed point (sums of float32 weights are exact in float64)."""
    n, k, T, D = 48, 12, 30, 3
    net = inp.network(n=n, k_in=k, seed=seed)
    st, ix = inp.spike_raster(n, T, 5, seed + 10)
    sE, sI = oracle.route(n, T, D, net["row_ptr"], net["col"], net["w"], net["inh"], st, ix)
    W = _dense(n, net["row_ptr"], net["col"], net["w"].astype(np.float64))
    exc = net["inh"] == 0
    for t in range(T):
        s = np.zeros(n)
        if t - D >= 0:
            s[ix[st == t - D]] = 1.0
        refE = W @ (s * exc)
        refI = W @ (s * ~exc)
        for got, ref in ((sE[t], refE), (sI[t], refI)):
            a = got * 2.0**32
            b = ref * 2.0**32
            assert np.array_equal(a, np.round(a)) and np.array_equal(a, b)


def _no_input_net(n, V0):
    return {"row_ptr": np.zeros(n + 1, np.int64), "col": np.zeros(0, np.int32),
            "w": np.zeros(0, np.float32), "inh": np.zeros(n, np.uint8), "V0": V0}


def test_network_without_synapses_equals_independent():
    V0 = np.linspace(-70, -60, 6)
    I = np.linspace(0, 15, 6)
    a = oracle.simulate_network(HH, _no_input_net(6, V0), 3000, 0.025, 40, SYN, I=I,
                                trace_idx=np.arange(6))
    b = oracle.simulate(HH, I, V0, 3000, 0.025)
    assert np.array_equal(a["V"], b["V"])
    assert np.array_equal(a["counts"], b["counts"])


@pytest.mark.parametrize("inhibitory", [0, 1])
def test_delay_onset_and_sign(inhibitory):
    """A single forced spike of neuron 0 at step s reaches neuron 1 exactly at
    step s + D: V_1 is untouched before, moves toward E_E (up) or E_I (down)
    from that step on."""
    s, D, T = 5, 7, 40
    net = {"row_ptr": np.array([0, 0, 1], np.int64), "col": np.array([0], np.int32),
           "w": np.array([5.0], np.float32), "inh": np.array([inhibitory, 0], np.uint8),
           "V0": np.array([-65.0, -65.0])}
    base = oracle.simulate_network(PASSIVE, net, T, 0.025, D, SYN,
                                   forced=(np.zeros(0), np.zeros(0)), trace_idx=[1])
    hit = oracle.simulate_network(PASSIVE, net, T, 0.025, D, SYN,
                                  forced=(np.array([s]), np.array([0])), trace_idx=[1])
    dv = hit["V"][:, 0] - base["V"][:, 0]
    assert np.all(dv[: s + D] == 0.0)
    assert (dv[s + D] > 0) if not inhibitory else (dv[s + D] < 0)


def test_passive_synapse_matches_ode():
    """Passive membrane receiving one excitatory event of w nS at t0:
    C dV/dt = -gL (V - EL) - g(t)(V - E_E), g(t) = w 1e-6/A e^{-(t-t0)/tau_E}.
    The oracle at dt = 1e-3 ms follows an adaptive RK solution within 1e-3 mV
    (pins the unit conversion, the decay constant and E_E)."""
    integ = pytest.importorskip("scipy.integrate")
    dt, D, T = 0.001, 1000, 30_000
    w = 2.0
    net = {"row_ptr": np.array([0, 0, 1], np.int64), "col": np.array([0], np.int32),
           "w": np.array([w], np.float32), "inh": np.array([0, 0], np.uint8),
           "V0": np.array([-65.0, -65.0])}
    r = oracle.simulate_network(PASSIVE, net, T, dt, D, SYN,
                                forced=(np.array([0]), np.array([0])), trace_idx=[1])
    t0 = D * dt
    g0 = float(np.float32(w)) * 1e-6 / SYN["area_cm2"]

    def rhs(t, y):
        g = g0 * math.exp(-(t - t0) / SYN["tau_E"]) if t >= t0 else 0.0
        return [(-0.1 * (y[0] + 65.0) - g * (y[0] - 0.0)) / 1.0]

    ts = (np.arange(T) + 1) * dt
    sol = integ.solve_ivp(rhs, (t0, ts[-1]), [-65.0], t_eval=ts[D:], rtol=1e-11,
                          atol=1e-12, method="DOP853", max_step=0.01)
    err = np.abs(r["V"][D:, 0] - sol.y[0])
    assert sol.y[0].max() > -64.0   # a visible EPSP
    assert err.max() < 1e-3


def _brute_force_network(model, net, T, dt, D, syn, bg, I, seed):
    """Tiny closed-loop network with dense weights and an explicit list of
    pending events (no ring buffer, no CSR), stepping neurons with the
    oracle's single-neuron update."""
    n = net["V0"].size
    W = _dense(n, net["row_ptr"], net["col"], net["w"].astype(np.float64))
    V = net["V0"].astype(np.float64).copy()
    P, Ca = [], []
    for i in range(n):
        p, c = oracle.init_neuron(model, V[i])
        P.append(p)
        Ca.append(c)
    gE = np.zeros(n)
    gI = np.zeros(n)
    pending = []   # (arrival step, pre)
    thr = oracle.poisson_table(oracle.background_lambda(bg["K"], bg["rate_hz"], dt)) \
        if bg else None
    to_mS = 1e-6 / syn["area_cm2"]
    spikes = []
    Vtr = np.zeros((T, n))
    for t in range(T):
        arriving = [j for (a, j) in pending if a == t]
        pending = [(a, j) for (a, j) in pending if a != t]
        for j in arriving:
            if net["inh"][j]:
                gI += W[:, j]
            else:
                gE += W[:, j]
        for i in range(n):
            if thr is not None:
                k = oracle.poisson_sample(oracle.background_word(seed, t, i), thr)
                gE[i] += k * bg["w"]
        new = []
        for i in range(n):
            Vn, P[i], Ca[i] = oracle.step_neuron(model, V[i], P[i], Ca[i], dt, I[i],
                                                 gE[i] * to_mS, syn["E_E"],
                                                 gI[i] * to_mS, syn["E_I"])
            if V[i] < 0.0 <= Vn:
                new.append(i)
                spikes.append((t, i))
            V[i] = Vn
        for i in new:
            pending.append((t + D, i))
        gE *= math.exp(-dt / syn["tau_E"])
        gI *= math.exp(-dt / syn["tau_I"])
        Vtr[t] = V
    return Vtr, spikes


def test_closed_loop_matches_brute_force():
    """Ring buffer + CSR + background closed loop == brute force with dense
    weights and an event list, bit for bit, on a 12-neuron network."""
    n, T, D, dt = 12, 600, 4, 0.025
    net = inp.network(n=n, k_in=5, seed=3, mu=1.5, sigma=0.5)
    I = np.linspace(2.0, 9.0, n)
    bg = {"rate_hz": 5.0, "K": 400, "w": 3.0}
    r = oracle.simulate_network(HH, net, T, dt, D, SYN, bg=bg, I=I, seed=11,
                                trace_idx=np.arange(n))
    Vb, sp = _brute_force_network(HH, net, T, dt, D, SYN, bg, I, 11)
    assert len(sp) > 5
    assert np.array_equal(r["V"], Vb)
    got = sorted((int(r["spk_step"][i][k]), i) for i in range(n) for k in range(r["counts"][i]))
    assert got == sorted(sp)


def test_per_step_current_in_network():
    """Per-step currents in the network oracle (the sinusoidal drive's
    input path): with no synapses a network run with I_steps [T][N] equals the
    independent-neuron oracle given the same I_steps, bit for bit, and a
    constant I_steps equals the constant-current run."""
    rng = np.random.default_rng(8)
    N, T, dt = 12, 800, 0.01
    V0 = rng.uniform(-70, -60, N).astype(np.float32)
    Is = oracle.sin_drive_steps(rng.uniform(0, 15, N), rng.uniform(5, 300, N).astype(np.float32),
                                np.zeros(N, np.float32), dt, T) + 3.0
    net = {"row_ptr": np.zeros(N + 1, np.int64), "col": np.zeros(0, np.int32), "w": np.zeros(0),
           "inh": np.zeros(N, np.uint8), "V0": V0}
    syn = {"tau_E": 5.0, "tau_I": 10.0, "E_E": 0.0, "E_I": -80.0, "area_cm2": 2e-4}
    a = oracle.simulate_network(HH, net, T, dt, 2, syn, I_steps=Is, trace_idx=np.arange(N))
    b = oracle.simulate(HH, np.zeros(N), V0, T, dt, I_steps=Is)
    assert np.array_equal(a["V"], b["V"]) and np.array_equal(a["counts"], b["counts"])
    assert a["counts"].sum() > 0
    c = oracle.simulate_network(HH, net, T, dt, 2, syn, I_steps=np.full((T, N), 4.0), trace_idx=np.arange(N))
    d = oracle.simulate_network(HH, net, T, dt, 2, syn, I=np.full(N, 4.0), trace_idx=np.arange(N))
    assert np.array_equal(c["V"], d["V"])
