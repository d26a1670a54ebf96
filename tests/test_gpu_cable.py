"""GPU parity of the multi-compartment cells (hh_net_desc.morph: a soma and
three dendrites per warp, the cable term by the explicit second difference)
against the FP64 multi-compartment oracle on the same compartment tree:
spike counts and times of every compartment, the V traces, somatic
responses to purely dendritic input; no coupling reduces to point neurons
bit for bit; the window kernels (a network) carry the same coupling."""
import numpy as np
import pytest

import oracle
from paper_2601_21407_gb300 import hh, inputs as inp

from test_gpu_neurons import T_TOL_MS, spike_time_errors

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _run(c, T, dt, prec, morph=True, csr=None, trace=True):
    torch = _torch()
    N = c["V0"].size
    kw = {}
    if csr is not None:
        kw = dict(csr=csr, inh=np.zeros(N, np.uint8), delay_steps=20,
                  syn={"tau_E": 5.0, "tau_I": 10.0, "E_E": 0.0, "E_I": -80.0, "area_cm2": 2e-4})
    net = hh.Network(c["V0"], dt, I_const=c["I"], precision=prec, morph=c["morph"] if morph else None, **kw)
    net.set_channels(0, inp.CLASSIC_HH, gbar=c["gbar"])
    rec, b = hh.make_record(N, T, trace=N if trace else 0, spike_cap=200 * N)
    net.step(T, rec=rec)
    torch.cuda.synchronize()
    out = {"counts": b["counts"].cpu().numpy(), "spk": hh.spikes_to_numpy(b),
           "status": int(net.readout(hh.HH_READ_STATUS)[0])}
    if trace:
        out["V"] = b["V_trace"].cpu().numpy()
    net.close()
    return out


@pytest.mark.parametrize("prec", [hh.HH_PREC_FAST, hh.HH_PREC_ACCURATE])
def test_cable_matches_oracle(prec):
    """64 cells (soma + 3 dendrites x 8 compartments, active dendrites at a
    third of the somatic Na/K densities, g_axial 2 mS/cm^2, soma 4x the area),
    stimulated at the soma, a distal dendrite or both, 30 ms at dt 0.01 ms:
    identical spike counts in every compartment, spike times within 0.05 ms,
    |dV| below 0.1 mV for 90 % of compartments; cells driven only at a
    distal dendrite fire at the soma."""
    c = inp.cable_cells(64, seed=1)
    T, dt = 3000, 0.01
    g = _run(c, T, dt, prec)
    ref = oracle.simulate_cable(inp.CLASSIC_HH, c["parent"], c["area"], c["morph"]["g_axial"], c["I"], c["V0"],
                                T, dt, gbar=c["gbar"], spk_cap=64)
    assert g["status"] == 0
    assert np.array_equal(g["counts"], ref["counts"])
    errs = spike_time_errors(g, ref, dt)
    dV = np.abs(g["V"] - ref["V"]).max(0)
    print(f"prec {prec}: compartments spiking {int((ref['counts'] > 0).sum())}, spike-time max "
          f"{max(errs.values()):.2e} ms, |dV| median {np.median(dV):.2e} p90 {np.quantile(dV, 0.9):.2e} mV")
    assert max(errs.values()) <= T_TOL_MS
    assert np.quantile(dV, 0.9) < 0.1
    soma = np.arange(64) * 32
    dendritic_only = soma[c["I"][soma] == 0.0]
    assert dendritic_only.size > 5 and (ref["counts"][dendritic_only] > 0).mean() > 0.5


def test_cable_without_coupling_is_point_neurons():
    """g_axial = 0: the cells' compartments are the point neurons of the same
    arrays, bit for bit."""
    c = inp.cable_cells(16, seed=2, g_axial=0.0)
    a = _run(c, 2000, 0.01, hh.HH_PREC_FAST)
    b = _run(c, 2000, 0.01, hh.HH_PREC_FAST, morph=False)
    assert np.array_equal(a["V"], b["V"]) and np.array_equal(a["counts"], b["counts"])


def test_cable_in_window_kernels():
    """The same cells as a network whose synapses all have weight 0 run on
    the window kernels (a launch per 10 steps, routing between): the traces
    equal the independent-cell kernel's to 1e-3 mV and the counts exactly."""
    c = inp.cable_cells(32, seed=3)
    N = c["V0"].size
    rng = np.random.default_rng(0)
    row_ptr = np.arange(0, (N + 1) * 4, 4, dtype=np.int64)
    col = rng.integers(0, N, N * 4).astype(np.int32)
    w = np.zeros(N * 4, np.float32)
    a = _run(c, 2000, 0.01, hh.HH_PREC_FAST)
    b = _run(c, 2000, 0.01, hh.HH_PREC_FAST, csr=(row_ptr, col, w))
    assert np.array_equal(a["counts"], b["counts"]) and a["counts"].sum() > 0
    assert np.abs(a["V"] - b["V"]).max() <= 1e-3


def test_cable_rejects_bad_morphology():
    c = inp.cable_cells(2, seed=0)
    with pytest.raises(hh.HHError) as e:
        hh.Network(c["V0"][:40], 0.01, morph=c["morph"])  # not a multiple of 32
    assert e.value.status == hh.HH_EINVAL
    bad = dict(c["morph"], n_per_dendrite=11)  # 1 + 3 x 11 > 32
    with pytest.raises(hh.HHError):
        hh.Network(c["V0"], 0.01, morph=bad)
