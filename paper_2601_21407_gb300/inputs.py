"""Seeded synthetic inputs and neuron-model tables for the HH hot path.

This module is shared by the CUDA path, the FP64 oracle's tests and the
benchmark.  It holds parameters and random draws only -- none of the method's
arithmetic (no rate function, no integrator, no routing).  Every array that is
handed to both sides is produced here once, in the precision the library
consumes (float32 / int32), and the oracle reads the very same values.

Neuron models are plain data: a list of channels, each with a reversal
potential E_X, a maximal conductance gbar_X and a list of gates with an
exponent, following the general form I = C_m dV/dt + sum_X gbar_X eta_X(p)(V-E_X)
with dp/dt = alpha_p(V)(1-p) - beta_p(V) p (Methods, Eq. hh_eq_full), where
eta_X is the product of the gates raised to their exponents.

A rate function is a tuple (form, a, vh, k[, vh2, k2, c]) evaluated as
c + form(V):
  const   : a
  exp     : a * exp((V - vh)/k)
  sigmoid : a / (1 + exp((V - vh)/k))
  linoid  : a * (V - vh) / (1 - exp(-(V - vh)/k))      (removable point at V = vh)
  bell    : a / (exp((V - vh)/k) + exp((V - vh2)/k2))
Gate kinds:
  ab      : f1 = alpha(V), f2 = beta(V)                       [1/ms]
  inftau  : f1 = p_inf(V), f2 = tau(V)                        [-, ms]
  ca      : p_inf = Ca / (Ca + f1.a), tau = f2(V)              (Ca in uM)
"""
from __future__ import annotations

import math
import numpy as np

# ---------------------------------------------------------------------------
# Model tables
# ---------------------------------------------------------------------------


def fn(form, a, vh=0.0, k=1.0, vh2=0.0, k2=1.0, c=0.0):
    return (form, float(a), float(vh), float(k), float(vh2), float(k2), float(c))


# Classic squid-axon HH (Hodgkin & Huxley 1952, Methods "HH point neuron"),
# modern convention with rest near -65 mV.  Rate constants are the textbook
# set; reversal potentials and maximal conductances are the ones the
# single-neuron workload names (ENa=50, EK=-77, EL=-54.4 mV; 120/36/0.3 mS/cm^2).
CLASSIC_HH = {
    "name": "hh1952",
    "C_m": 1.0,  # uF/cm^2
    "channels": [
        {"name": "Na", "E": 50.0, "gbar": 120.0, "gates": [
            {"kind": "ab", "power": 3, "f1": fn("linoid", 0.1, -40.0, 10.0),
             "f2": fn("exp", 4.0, -65.0, -18.0)},                  # m
            {"kind": "ab", "power": 1, "f1": fn("exp", 0.07, -65.0, -20.0),
             "f2": fn("sigmoid", 1.0, -35.0, -10.0)},              # h
        ]},
        {"name": "K", "E": -77.0, "gbar": 36.0, "gates": [
            {"kind": "ab", "power": 4, "f1": fn("linoid", 0.01, -55.0, 10.0),
             "f2": fn("exp", 0.125, -65.0, -80.0)},                # n
        ]},
        {"name": "L", "E": -54.4, "gbar": 0.3, "gates": []},
    ],
    "calcium": None,
}

# Multi-channel point neuron: Na, Kdr (the HH pair above), a fast transient
# K current KA (a^3 b), a high-voltage-activated L-type Ca current (s^2,
# ohmic, E_Ca = 120 mV), a Ca-dependent K current KCa and a hyperpolarisation
# activated cation current Ih, with a first-order Ca pool
#   d[Ca]/dt = -k_Ca * I_Ca - ([Ca] - Ca_rest)/tau_Ca.
# The kinetic forms follow the shapes used for these currents in the
# thalamic / cortical models of Huguenard & McCormick (1992; I_A, I_h) and
# Traub et al. (1991; I_Ca); the maximal conductances are chosen so that the
# neuron stays excitable and fires repetitively over 0-15 uA/cm^2.  The table
# is a workload definition: both the oracle and the CUDA path consume it.
MULTI_CHANNEL = {
    "name": "multi6",
    "C_m": 1.0,
    "channels": [
        {"name": "Na", "E": 50.0, "gbar": 120.0, "gates": [
            {"kind": "ab", "power": 3, "f1": fn("linoid", 0.1, -40.0, 10.0),
             "f2": fn("exp", 4.0, -65.0, -18.0)},
            {"kind": "ab", "power": 1, "f1": fn("exp", 0.07, -65.0, -20.0),
             "f2": fn("sigmoid", 1.0, -35.0, -10.0)},
        ]},
        {"name": "Kdr", "E": -77.0, "gbar": 36.0, "gates": [
            {"kind": "ab", "power": 4, "f1": fn("linoid", 0.01, -55.0, 10.0),
             "f2": fn("exp", 0.125, -65.0, -80.0)},
        ]},
        {"name": "KA", "E": -77.0, "gbar": 2.0, "gates": [
            {"kind": "inftau", "power": 3, "f1": fn("sigmoid", 1.0, -60.0, -8.5),
             "f2": fn("bell", 1.0, -35.8, 19.7, -79.7, -12.7, c=0.37)},
            {"kind": "inftau", "power": 1, "f1": fn("sigmoid", 1.0, -78.0, 6.0),
             "f2": fn("bell", 1.0, -46.0, 5.0, -238.0, -37.5, c=19.0)},
        ]},
        {"name": "CaL", "E": 120.0, "gbar": 0.2, "gates": [
            {"kind": "ab", "power": 2, "f1": fn("sigmoid", 1.6, 5.0, -13.888889),
             "f2": fn("linoid", -0.02, -8.9, -5.0)},
        ]},
        {"name": "KCa", "E": -77.0, "gbar": 0.1, "gates": [
            {"kind": "ca", "power": 1, "f1": fn("const", 3.0),
             "f2": fn("const", 10.0)},
        ]},
        {"name": "Ih", "E": -43.0, "gbar": 0.2, "gates": [
            {"kind": "inftau", "power": 1, "f1": fn("sigmoid", 1.0, -75.0, 5.5),
             "f2": fn("bell", 1.0, -169.65, -11.628, 26.676, 14.265)},
        ]},
        {"name": "L", "E": -54.4, "gbar": 0.3, "gates": []},
    ],
    # Ca pool fed by the channel named "CaL"; Ca in uM, k_Ca in uM/ms per uA/cm^2
    "calcium": {"channel": "CaL", "tau": 20.0, "k": 0.05, "rest": 0.05},
}

def _bc2008(name, gNa, gKd, gM, gL, EL, VT, tau_max):
    """Pospischil et al. 2008 minimal HH-type cortical neuron (Traub-Miles Na
    and delayed-rectifier K with threshold shift V_T, a slow M-type K current
    p with p_inf = 1/(1 + e^{-(V+35)/10}) and tau_p = tau_max/(3.3 e^{(V+35)/20}
    + e^{-(V+35)/20}), leak), in the closed forms of this table: the Traub
    rates are linoid / exp / sigmoid forms with half-points shifted by V_T,
    and 3.3 e^{x/20} = e^{(x + 20 ln 3.3)/20} puts tau_p in the bell form."""
    return {
        "name": name, "C_m": 1.0,
        "channels": [
            {"name": "Na", "E": 50.0, "gbar": gNa, "gates": [
                {"kind": "ab", "power": 3, "f1": fn("linoid", 0.32, VT + 13.0, 4.0),
                 "f2": fn("linoid", -0.28, VT + 40.0, -5.0)},
                {"kind": "ab", "power": 1, "f1": fn("exp", 0.128, VT + 17.0, -18.0),
                 "f2": fn("sigmoid", 4.0, VT + 40.0, -5.0)},
            ]},
            {"name": "Kd", "E": -90.0, "gbar": gKd, "gates": [
                {"kind": "ab", "power": 4, "f1": fn("linoid", 0.032, VT + 15.0, 5.0),
                 "f2": fn("exp", 0.5, VT + 10.0, -40.0)},
            ]},
            {"name": "M", "E": -90.0, "gbar": gM, "gates": [
                {"kind": "inftau", "power": 1, "f1": fn("sigmoid", 1.0, -35.0, -10.0),
                 "f2": fn("bell", tau_max, -35.0 - 20.0 * math.log(3.3), 20.0, -35.0, -20.0)},
            ]},
            {"name": "L", "E": EL, "gbar": gL, "gates": []},
        ],
        "calcium": None,
    }


# Regular-spiking pyramidal and fast-spiking interneuron parameter sets of the
# BC2008 model (the cortex variant's excitatory and inhibitory cells).
BC2008_RS = _bc2008("bc2008_rs", 56.0, 6.0, 0.075, 0.0205, -70.3, -56.2, 608.0)
BC2008_FS = _bc2008("bc2008_fs", 58.0, 3.9, 0.0787, 0.038, -70.4, -57.9, 502.0)

MODELS = {"hh1952": CLASSIC_HH, "multi6": MULTI_CHANNEL, "bc2008_rs": BC2008_RS, "bc2008_fs": BC2008_FS}


def cortex_network(n=10_000, k_in=1_000, exc_frac=0.8, seed=0, w_mu=0.26, w_sd=0.026, g_inh=4.0):
    """The current-based cortex variant's stand-in network (the Potjans-
    Diesmann connection tables are not in this container): fixed in-degree
    k_in from distinct random sources, 80 % excitatory regular-spiking and
    20 % inhibitory fast-spiking BC2008 cells (model ids 0 / 1), synaptic
    current amplitudes ~ N(w_mu, w_sd) uA/cm^2 clipped at 0, inhibitory ones
    scaled by g_inh (their sign is that of the inhibitory current);
    V0 ~ U(-72, -66) mV."""
    gen = random_in_csr_fast if n * k_in > 2_000_000 else random_in_csr
    row_ptr, col, _ = gen(n, k_in, seed)
    rng = np.random.default_rng(seed + 7)
    n_exc = int(round(exc_frac * n))
    inh = np.zeros(n, np.uint8)
    inh[n_exc:] = 1
    w = np.clip(rng.normal(w_mu, w_sd, col.size), 0.0, None)
    w = np.where(inh[col] == 1, g_inh * w, w).astype(np.float32)
    return {"row_ptr": row_ptr, "col": col, "w": w, "inh": inh, "model_id": inh.copy(),
            "V0": rng.uniform(-72.0, -66.0, n).astype(np.float32), "n": n, "k_in": k_in}


def model_gbar(model) -> np.ndarray:
    return np.array([c["gbar"] for c in model["channels"]], dtype=np.float64)


# ---------------------------------------------------------------------------
# Seeded workload generators (numpy PCG64; seed 0 by default)
# ---------------------------------------------------------------------------


def single_neurons(n=1024, seed=0, i_max=20.0):
    """Independent classic HH neurons with constant injected current.

    I ~ U(0, i_max) uA/cm^2, V0 = -65 mV, gates at steady state at V0.
    Returns float32 arrays (the library's precision); the oracle reads the
    same float32 values widened to float64.
    """
    rng = np.random.default_rng(seed)
    I = rng.uniform(0.0, i_max, n).astype(np.float32)
    V0 = np.full(n, -65.0, dtype=np.float32)
    return {"I": I, "V0": V0}


def sin_sweep(n_f=256, n_A=256, f_min=1.0, f_max=1000.0, A_max=20.0, I0=0.0):
    """Frequency-response sweep of classic HH neurons under sinusoidal
    current (the filter-bank workload): one neuron per (frequency, amplitude)
    pair, frequencies log-spaced in [f_min, f_max] Hz, amplitudes uniform in
    (0, A_max] uA/cm^2, a constant bias I0, phase 0, V0 = -65 mV.  Neuron
    i = a * n_f + f.  float32 arrays."""
    f = np.geomspace(f_min, f_max, n_f)
    A = np.linspace(A_max / n_A, A_max, n_A)
    ff, AA = np.meshgrid(f, A)
    n = n_f * n_A
    return {"freq_hz": ff.reshape(-1).astype(np.float32), "amp": AA.reshape(-1).astype(np.float32),
            "phase": np.zeros(n, np.float32), "I": np.full(n, I0, np.float32),
            "V0": np.full(n, -65.0, np.float32), "n_f": n_f, "n_A": n_A}


CABLE_LANES = 32


def cable_cells(n_cells, n_dend=3, n_per=8, seed=0, g_axial=2.0, soma_area_ratio=4.0,
                dend_scale=1.0 / 3.0):
    """Multi-compartment cells of the classic HH channels (the morphology
    workload: a soma and three dendrites), laid out 32 compartments per cell:
    index 32 k the soma of cell k, 32 k + 1 + d n_per + j compartment j of
    dendrite d, the remaining lanes passive and unstimulated.  Somata carry the
    full channel densities, dendrites dend_scale of the Na and K densities.
    Each cell is stimulated, by a constant current U(5, 40) uA/cm^2, at its
    soma, at the last compartment of a random dendrite, or at both.  Returns
    V0, I, gbar [3][N] (float32), the parent index and relative area of every
    compartment (-1 and 1 for the idle lanes) and the morphology."""
    rng = np.random.default_rng(seed)
    L = CABLE_LANES
    n_comp = 1 + n_dend * n_per
    assert n_comp <= L
    N = n_cells * L
    g0 = model_gbar(CLASSIC_HH).astype(np.float32)
    gbar = np.zeros((3, N), np.float32)
    parent = np.full(N, -1, np.int64)
    area = np.ones(N)
    I = np.zeros(N, np.float32)
    for k in range(n_cells):
        b = k * L
        gbar[:, b] = g0
        area[b] = soma_area_ratio
        for d in range(n_dend):
            for j in range(n_per):
                c = b + 1 + d * n_per + j
                parent[c] = b if j == 0 else c - 1
                gbar[:, c] = g0 * np.array([dend_scale, dend_scale, 1.0], np.float32)
        gbar[2, b + n_comp: b + L] = g0[2]  # idle lanes: leak only
        where = rng.integers(0, 3)
        amp = rng.uniform(5.0, 40.0)
        if where in (0, 2):
            I[b] = amp
        if where in (1, 2):
            I[b + 1 + int(rng.integers(0, n_dend)) * n_per + n_per - 1] = amp
    return {"V0": np.full(N, -65.0, np.float32), "I": I, "gbar": gbar, "parent": parent, "area": area,
            "morph": {"n_dendrites": n_dend, "n_per_dendrite": n_per, "g_axial": g_axial,
                      "soma_area_ratio": soma_area_ratio}, "n_cells": n_cells, "n_comp": n_comp}


def multi_channel_neurons(n=1_000_000, seed=0, sigma=0.3, i_max=15.0,
                          model=MULTI_CHANNEL):
    """Independent multi-channel neurons with per-neuron maximal conductances.

    gbar[c][i] = gbar_std[c] * LogNormal(0, sigma); I ~ U(0, i_max).
    Returns gbar as float32 [n_channels][n].
    """
    rng = np.random.default_rng(seed)
    g0 = model_gbar(model)
    gbar = (g0[:, None] * rng.lognormal(0.0, sigma, (len(g0), n))).astype(np.float32)
    I = rng.uniform(0.0, i_max, n).astype(np.float32)
    V0 = np.full(n, -65.0, dtype=np.float32)
    return {"I": I, "V0": V0, "gbar": gbar}


def random_in_csr(n, k_in, seed, mu=-1.0, sigma=0.5, n_pre=None, allow_self=False):
    """Fixed in-degree random graph as an in-CSR (rows = postsynaptic neuron).

    Each row draws k_in distinct presynaptic sources uniformly from the other
    n-1 neurons (no self-loops), sorted ascending; weights ~ LogNormal(mu, sigma)
    in nS, float32.  Returns row_ptr (int64 [n+1]), col_idx (int32), weight
    (float32).
    """
    rng = np.random.default_rng(seed)
    n_pre = n if n_pre is None else n_pre
    k_in = int(k_in)
    pool = n_pre - (0 if allow_self else 1)
    if k_in > pool:
        raise ValueError("in-degree larger than the number of possible sources")
    cols = np.empty((n, k_in), dtype=np.int32)
    for i in range(n):
        c = rng.choice(pool, size=k_in, replace=False)
        if not allow_self:
            c = c + (c >= i)
        c.sort()
        cols[i] = c
    w = rng.lognormal(mu, sigma, n * k_in).astype(np.float32)
    row_ptr = np.arange(0, (n + 1) * k_in, k_in, dtype=np.int64)
    return row_ptr, cols.reshape(-1), w


def random_in_csr_fast(n, k_in, seed, mu=-1.0, sigma=0.5):
    """Same distribution as random_in_csr (k_in distinct non-self sources per
    row, sorted) generated block-wise with sort-based rejection of duplicates;
    used for the 1e8-synapse network where a per-row loop is too slow.  The two
    generators draw different random streams."""
    rng = np.random.default_rng(seed)
    k_in = int(k_in)
    cols = np.empty((n, k_in), dtype=np.int32)
    block = max(1, min(n, (1 << 24) // max(k_in, 1)))
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        rows = r1 - r0
        extra = max(8, int(k_in * k_in / max(n - 1, 1) * 3) + 8)
        done = np.zeros(rows, dtype=bool)
        out = cols[r0:r1]
        while not done.all():
            idx = np.nonzero(~done)[0]
            cand = rng.integers(0, n - 1, size=(idx.size, k_in + extra), dtype=np.int64)
            cand = cand + (cand >= (r0 + idx)[:, None])
            cand.sort(axis=1)
            dup = np.zeros_like(cand, dtype=bool)
            dup[:, 1:] = cand[:, 1:] == cand[:, :-1]
            n_unique = (~dup).sum(axis=1)
            ok = n_unique >= k_in
            for j in np.nonzero(ok)[0]:
                u = cand[j][~dup[j]]
                # keep a uniformly random subset of the distinct candidates
                sel = rng.choice(u.size, size=k_in, replace=False)
                sel.sort()
                out[idx[j]] = u[sel]
            done[idx[ok]] = True
    w = rng.lognormal(mu, sigma, n * k_in).astype(np.float32)
    row_ptr = np.arange(0, (n + 1) * k_in, k_in, dtype=np.int64)
    return row_ptr, cols.reshape(-1), w


def random_in_csr_vec(n, k_in, seed, mu=-1.0, sigma=0.5):
    """Same distribution as random_in_csr (k_in distinct non-self sources per
    row, sorted), fully vectorised: per block of rows, k_in + extra
    candidates are drawn, sorted and de-duplicated, each distinct candidate
    gets a uniform random key and the k_in smallest keys are kept (a uniform
    subset); rows with fewer than k_in distinct candidates are drawn again.
    For sparse rows (k_in well below n); draws its own random stream."""
    rng = np.random.default_rng(seed)
    k_in = int(k_in)
    cols = np.empty((n, k_in), dtype=np.int32)
    extra = max(8, int(k_in * k_in / max(n - 1, 1) * 3) + 8)
    block = max(1, min(n, (1 << 22) // (k_in + extra)))
    for r0 in range(0, n, block):
        rows = np.arange(r0, min(n, r0 + block))
        while rows.size:
            cand = rng.integers(0, n - 1, size=(rows.size, k_in + extra), dtype=np.int64)
            cand += cand >= rows[:, None]
            cand.sort(axis=1)
            dup = np.zeros(cand.shape, dtype=bool)
            dup[:, 1:] = cand[:, 1:] == cand[:, :-1]
            ok = (~dup).sum(axis=1) >= k_in
            keys = rng.random(cand.shape)
            keys[dup] = 2.0
            sel = np.argpartition(keys, k_in - 1, axis=1)[:, :k_in]
            pick = np.take_along_axis(cand, sel, axis=1)
            pick.sort(axis=1)
            cols[rows[ok]] = pick[ok]
            rows = rows[~ok]
    w = rng.lognormal(mu, sigma, n * k_in).astype(np.float32)
    row_ptr = np.arange(0, (n + 1) * k_in, k_in, dtype=np.int64)
    return row_ptr, cols.reshape(-1), w


def network(n=38_000, k_in=2_632, exc_frac=0.8, seed=0, mu=-1.0, sigma=0.5,
            fast=None):
    """Sparse conductance-based HH network (in-CSR by postsynaptic neuron).

    Neurons 0 .. exc_frac*n-1 are excitatory, the rest inhibitory; V0 ~ U(-70,-60).
    """
    if fast is None:
        fast = n * k_in > 2_000_000
    gen = random_in_csr_fast if fast else random_in_csr
    row_ptr, col, w = gen(n, k_in, seed, mu, sigma)
    rng = np.random.default_rng(seed + 1_000_003)
    n_exc = int(round(exc_frac * n))
    inh = np.zeros(n, dtype=np.uint8)
    inh[n_exc:] = 1
    V0 = rng.uniform(-70.0, -60.0, n).astype(np.float32)
    return {"row_ptr": row_ptr, "col": col, "w": w, "inh": inh, "V0": V0,
            "n": n, "k_in": k_in}


def spike_raster(n, n_steps, per_step, seed):
    """A synthetic spike raster for open-loop routing: `per_step` distinct
    presynaptic neurons drawn uniformly at every step.  Returns (step, idx)
    int32 arrays sorted by (step, idx)."""
    rng = np.random.default_rng(seed)
    steps, idx = [], []
    for t in range(n_steps):
        j = np.sort(rng.choice(n, size=per_step, replace=False)).astype(np.int32)
        steps.append(np.full(per_step, t, dtype=np.int32))
        idx.append(j)
    if not steps:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    return np.concatenate(steps), np.concatenate(idx)


def recurrent_layer(B=128, n_in=700, n_hid=1024, n_out=20, T=250, seed=0,
                    dt_outer_ms=0.1, rate_max_hz=50.0, w_in_scale=None,
                    w_rec_scale=None, i_bias=4.0):
    """Differentiable recurrent HH layer workload (shape of a spoken-digit task).

    X[t, b, c] ~ Bernoulli(rate_c * dt_outer) with rate_c ~ U(0, rate_max) Hz;
    weights in uA/cm^2 per input spike, rounded to bfloat16-representable
    float32 values (the tensor-core path stores them in bf16 exactly);
    labels ~ U{0..n_out-1}.
    """
    rng = np.random.default_rng(seed)
    rate = rng.uniform(0.0, rate_max_hz, n_in)
    p = rate * dt_outer_ms * 1e-3
    X = (rng.random((T, B, n_in)) < p[None, None, :]).astype(np.float32)
    if w_in_scale is None:
        w_in_scale = 40.0
    if w_rec_scale is None:
        w_rec_scale = 2.0
    W_in = to_bf16_exact(rng.normal(0.0, w_in_scale / math.sqrt(n_in), (n_in, n_hid)))
    W_rec = to_bf16_exact(rng.normal(0.0, w_rec_scale / math.sqrt(n_hid), (n_hid, n_hid)))
    W_out = (rng.normal(0.0, 1.0 / math.sqrt(n_hid), (n_out, n_hid))).astype(np.float32)
    bias = np.full(n_hid, i_bias, dtype=np.float32)
    labels = rng.integers(0, n_out, B).astype(np.int32)
    return {"X": X, "W_in": W_in, "W_rec": W_rec, "W_out": W_out, "bias": bias,
            "labels": labels}


def to_bf16_exact(a) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (ties to even) and return
    them as float32, so that a bf16 copy holds exactly the same numbers."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _batched_net(task):
    """Worker of batched_networks: one network's in-CSR (columns shifted to
    the concatenated index) written into the shared output arrays."""
    from multiprocessing import shared_memory
    n, ki, seed, mu, sigma, off, nnz0, names = task
    gen = random_in_csr_vec if n * ki > 2_000_000 else random_in_csr
    _, c, w = gen(n, ki, seed, mu, sigma)
    if names is None:
        return c + off, w
    sc, sw = shared_memory.SharedMemory(name=names[0]), shared_memory.SharedMemory(name=names[1])
    try:
        np.ndarray((c.size,), np.int32, sc.buf, offset=nnz0 * 4)[:] = c + off
        np.ndarray((w.size,), np.float32, sw.buf, offset=nnz0 * 4)[:] = w
    finally:
        sc.close()
        sw.close()
    return None


def batched_networks(n_nets=64, n_min=1_000, n_max=50_000, k_min=100, k_max=1_000,
                     seed=0, exc_frac=0.8, mu=-1.0, sigma=0.5, workers=1):
    """Many independent networks concatenated block-diagonally.

    Sizes ~ LogUniform(n_min, n_max), in-degree ~ U{k_min..k_max} (clipped to
    n-1), half of the networks use the classic HH model and half the
    multi-channel model (model id per neuron).  Returns a single in-CSR over the
    concatenated neuron index, net offsets and per-neuron model ids.  The
    networks' graphs are drawn from per-network seeds, so `workers` > 1
    (processes started with spawn, writing into shared memory) gives the
    same arrays as one process.
    """
    import multiprocessing as mp
    from multiprocessing import shared_memory
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_nets)).astype(np.int64)
    kin = rng.integers(k_min, k_max + 1, n_nets)
    kin = np.minimum(kin, sizes - 1)
    model_of_net = rng.integers(0, 2, n_nets).astype(np.uint8)
    offsets = np.zeros(n_nets + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    seeds = [int(rng.integers(0, 2**31)) for _ in range(n_nets)]
    nnz = sizes * kin
    nnz0 = np.zeros(n_nets + 1, dtype=np.int64)
    nnz0[1:] = np.cumsum(nnz)
    total = int(nnz0[-1])
    inh = np.zeros(int(offsets[-1]), np.uint8)
    model_id = np.zeros(int(offsets[-1]), np.uint8)
    for k in range(n_nets):
        n_exc = int(round(exc_frac * int(sizes[k])))
        inh[offsets[k] + n_exc: offsets[k + 1]] = 1
        model_id[offsets[k]: offsets[k + 1]] = model_of_net[k]
    row_ptr = np.zeros(int(offsets[-1]) + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.repeat(kin, sizes))
    if workers > 1:
        sc = shared_memory.SharedMemory(create=True, size=max(4, total * 4))
        sw = shared_memory.SharedMemory(create=True, size=max(4, total * 4))
        try:
            tasks = [(int(sizes[k]), int(kin[k]), seeds[k], mu, sigma, int(offsets[k]), int(nnz0[k]),
                      (sc.name, sw.name)) for k in range(n_nets)]
            order = sorted(range(n_nets), key=lambda k: -int(nnz[k]))  # largest first
            with mp.get_context("spawn").Pool(workers) as pool:
                pool.map(_batched_net, [tasks[k] for k in order], chunksize=1)
            col = np.ndarray((total,), np.int32, sc.buf).copy()
            w = np.ndarray((total,), np.float32, sw.buf).copy()
        finally:
            sc.close()
            sc.unlink()
            sw.close()
            sw.unlink()
    else:
        parts = [_batched_net((int(sizes[k]), int(kin[k]), seeds[k], mu, sigma, int(offsets[k]), 0, None))
                 for k in range(n_nets)]
        col = np.concatenate([p[0] for p in parts]).astype(np.int32)
        w = np.concatenate([p[1] for p in parts]).astype(np.float32)
    V0 = rng.uniform(-70.0, -60.0, int(offsets[-1])).astype(np.float32)
    return {"row_ptr": row_ptr, "col": col, "w": w, "inh": inh, "V0": V0,
            "offsets": offsets, "sizes": sizes, "k_in": kin, "model_id": model_id,
            "model_of_net": model_of_net}
