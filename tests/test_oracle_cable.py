"""Pins of the FP64 multi-compartment oracle (oracle.simulate_cable):
without axial coupling it is the point-neuron oracle bit for bit; a passive
tree under constant current settles to the solution of the linear
steady-state equations (the discrete cable with sealed ends), which pins the
signs, the area factors and the indexing of the explicit spatial term; and
identical dendrites stay identical."""
import numpy as np

import oracle
from paper_2601_21407_gb300 import inputs as inp

HH = inp.CLASSIC_HH


def star_of_chains(n_dend, n_per, soma_ratio):
    """Soma 0 and n_dend chains of n_per compartments, chain d's first
    compartment joined to the soma; areas 1 except the soma's."""
    parent = [-1]
    for d in range(n_dend):
        for j in range(n_per):
            parent.append(0 if j == 0 else len(parent) - 1)
    area = np.ones(len(parent))
    area[0] = soma_ratio
    return np.array(parent), area


def test_no_coupling_is_point_neurons():
    parent, area = star_of_chains(3, 4, 2.0)
    N = parent.size
    rng = np.random.default_rng(1)
    I = rng.uniform(0, 15, N)
    V0 = rng.uniform(-70, -60, N)
    a = oracle.simulate_cable(HH, parent, area, 0.0, I, V0, 2000, 0.01)
    b = oracle.simulate(HH, I, V0, 2000, 0.01)
    assert np.array_equal(a["V"], b["V"]) and np.array_equal(a["counts"], b["counts"])


def test_passive_tree_steady_state():
    """Leak-only compartments (g_L, E_L), current I0 into the soma: after 60
    membrane time constants every V equals the solution of
    g_L (V_c - E_L) = I_c + sum of the axial currents, to 1e-9 mV."""
    gL, EL, g_ax, r = 0.3, -54.4, 1.5, 3.0
    leak = {"name": "leak", "C_m": 1.0, "channels": [{"name": "L", "E": EL, "gbar": gL, "gates": []}],
            "calcium": None}
    parent, area = star_of_chains(3, 5, r)
    N = parent.size
    I = np.zeros(N)
    I[0] = 6.0
    I[7] = -2.0  # a second injection on dendrite 1
    T, dt = 20000, 0.01
    out = oracle.simulate_cable(leak, parent, area, g_ax, I, np.full(N, EL), T, dt, trace=True)
    A = np.zeros((N, N))
    b = I + gL * EL
    for c in range(N):
        A[c, c] += gL
    for c in range(1, N):
        p = parent[c]
        A[c, c] += g_ax
        A[c, p] -= g_ax
        A[p, p] += g_ax * area[c] / area[p]
        A[p, c] -= g_ax * area[c] / area[p]
    Vss = np.linalg.solve(A, b)
    assert np.abs(out["V"][-1] - Vss).max() < 1e-9
    assert Vss[0] > EL + 1.0 and Vss[7] < Vss[6]  # depolarised soma, the dendritic sink visible


def test_identical_dendrites_stay_identical():
    parent, area = star_of_chains(3, 6, 4.0)
    N = parent.size
    I = np.zeros(N)
    I[0] = 40.0
    out = oracle.simulate_cable(HH, parent, area, 2.0, I, np.full(N, -65.0), 3000, 0.01)
    V = out["V"]
    assert out["counts"][0] >= 2
    assert np.array_equal(V[:, 1:7], V[:, 7:13]) and np.array_equal(V[:, 1:7], V[:, 13:19])
