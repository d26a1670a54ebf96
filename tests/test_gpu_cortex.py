"""GPU parity of the current-based cortex variant (Methods, "Cerebral cortex
network"): BC2008 regular-spiking and fast-spiking cells, synapses that
inject their filtered currents (HH_SYN_CURRENT), dt 0.1 ms, a 1.5 ms delay
and the compound Poisson x Gaussian background, against the FP64 network
oracle on the same graph, counts and normals."""
import numpy as np
import pytest

import oracle
from paper_2601_21407_gb300 import hh, inputs as inp

pytestmark = pytest.mark.gpu

SYN = {"tau_E": 0.5, "tau_I": 0.5, "E_E": 0.0, "E_I": -80.0, "area_cm2": 2e-4}
BG = {"rate_hz": 8.0, "K": 2000, "w": 0.17, "sd": 0.017}


def _torch():
    import torch
    return torch


@pytest.mark.parametrize("prec", [hh.HH_PREC_FAST, hh.HH_PREC_ACCURATE])
def test_cortex_network_matches_oracle(prec):
    """2,000 cells (80 % RS, 20 % FS), in-degree 200, recurrent amplitudes
    N(0.26, 0.026) uA/cm^2 (inhibitory x 4), background 2,000 sources x 8 Hz
    x N(0.17, 0.017), 200 ms: V within 1e-2 mV of the oracle for the first
    10 ms, spike counts within +-1 for every cell over 50 ms and for >= 99 %
    over 200 ms, totals within 1 %."""
    torch = _torch()
    g = inp.cortex_network(n=2000, k_in=200, seed=1)
    T, dt, D = 2000, 0.1, 15
    net = hh.Network(g["V0"], dt, csr=(g["row_ptr"], g["col"], g["w"]), inh=g["inh"], syn=SYN, delay_steps=D,
                     bg=BG, seed=3, precision=prec, model_id=g["model_id"], syn_mode=hh.HH_SYN_CURRENT)
    net.set_channels(0, inp.BC2008_RS)
    net.set_channels(1, inp.BC2008_FS)
    rec, b = hh.make_record(2000, T, trace=2000, spike_cap=1_000_000)
    net.step(T, rec=rec)
    torch.cuda.synchronize()
    assert int(net.readout(hh.HH_READ_STATUS)[0]) == 0
    st, ix, _ = hh.spikes_to_numpy(b)
    V = b["V_trace"].cpu().numpy()
    net.close()
    ref = oracle.simulate_network([inp.BC2008_RS, inp.BC2008_FS], g, T, dt, D, SYN, bg=BG, seed=3,
                                  model_id=g["model_id"], syn_current=True, trace_idx=np.arange(2000))
    dv = np.abs(V[:100] - ref["V"][:100]).max()
    ss = ref["spk_step"]
    res = {}
    for t_ms in (50, 200):
        s_end = int(round(t_ms / dt))
        cg = np.bincount(ix[st < s_end], minlength=2000)
        cr = ((ss >= 0) & (ss < s_end)).sum(1)
        res[t_ms] = (np.abs(cg - cr), int(cg.sum()), int(cr.sum()))
    print(f"prec {prec}: V over 10 ms {dv:.2e} mV; 50 ms max diff {res[50][0].max()}; 200 ms within 1 "
          f"{(res[200][0] <= 1).mean():.4f} max {res[200][0].max()}, spikes {res[200][1]} vs {res[200][2]}")
    assert res[200][2] > 5000
    assert dv < 1e-2
    assert res[50][0].max() <= 1
    assert (res[200][0] <= 1).mean() >= 0.99
    assert abs(res[200][1] - res[200][2]) <= 0.01 * res[200][2]


def test_current_synapse_delivery_open_loop():
    """Open-loop routing in the current-based mode delivers the same fixed-
    point sums as in the conductance mode (the synapse model changes only
    how the neuron step uses them)."""
    torch = _torch()
    g = inp.cortex_network(n=500, k_in=50, seed=2)
    st, ix = inp.spike_raster(500, 30, 20, 4)
    out = []
    for mode in (hh.HH_SYN_CONDUCTANCE, hh.HH_SYN_CURRENT):
        net = hh.Network(g["V0"], 0.1, csr=(g["row_ptr"], g["col"], g["w"]), inh=g["inh"], syn=SYN,
                         delay_steps=15, syn_mode=mode)
        net.set_channels(0, inp.BC2008_RS)
        sE = torch.zeros((60, 500), dtype=torch.int64, device="cuda")
        sI = torch.zeros_like(sE)
        net.route_spikes(torch.as_tensor(st, device="cuda"), torch.as_tensor(ix, device="cuda"), 60, sE, sI)
        torch.cuda.synchronize()
        out.append((sE.cpu().numpy(), sI.cpu().numpy()))
        net.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][0].any() and out[0][1].any()


def test_cortex_rejects_bad_background_sd():
    g = inp.cortex_network(n=100, k_in=10, seed=0)
    with pytest.raises(hh.HHError) as e:
        hh.Network(g["V0"], 0.1, bg=dict(BG, sd=-1.0))
    assert e.value.status == hh.HH_EINVAL
