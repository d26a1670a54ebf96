"""GPU parity of the polynomial-rate path (HH_PREC_POLY: p_inf and
1 - e^{-dt/tau} of every gate from cubic tables fitted at hh_set_channels)
against the FP64 oracle, at the tolerances of the plain FP32 path: config 1
(1,024 classic neurons, 100 ms), config 4 (512 multi-channel neurons, 500 ms;
the full 1e6 population on sampled neurons), and the fallback to the SFU
arithmetic outside the tabulated range.  The closed-loop network in this
mode is one case of test_gpu_network.test_closed_loop_small_network."""
import numpy as np
import pytest

import oracle
from paper_2601_21407_gb300 import hh, inputs as inp

from test_gpu_neurons import T_TOL_MS, run_gpu, spike_time_errors

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def test_poly_tables_reported():
    """HH_READ_POLY gives each installed model's interval, first V and fit
    error, and nothing for the others."""
    x = inp.single_neurons(64, seed=0)
    net = hh.Network(x["V0"], 0.01, I_const=x["I"], precision=hh.HH_PREC_POLY,
                     model_id=np.array([0, 1] * 32, dtype=np.uint8))
    net.set_channels(0, inp.CLASSIC_HH)
    net.set_channels(1, inp.MULTI_CHANNEL)
    info = net.readout(hh.HH_READ_POLY).reshape(hh.HH_MAX_MODELS, 3)
    for k, m in ((0, inp.CLASSIC_HH), (1, inp.MULTI_CHANNEL)):
        h, v_lo, err, _ = hh.hh_poly_fit(m, 0.01)
        assert tuple(info[k]) == (np.float32(h), np.float32(v_lo), np.float32(err))
        assert err <= hh.HH_POLY_REL_ERR
    assert not info[2:].any()
    net.close()


def test_poly_rejects_table_kernels():
    x = inp.single_neurons(8, seed=0)
    with pytest.raises(hh.HHError) as e:
        hh.Network(x["V0"], 0.01, I_const=x["I"], precision=hh.HH_PREC_POLY, kernels=hh.HH_KERNELS_TABLE)
    assert e.value.status == hh.HH_EUNSUPPORTED


def test_poly_classic_population():
    """Config 1 (1,024 neurons, I ~ U(0, 20), dt 0.01 ms, 100 ms): identical
    spike counts, spike times within 0.05 ms for every neuron, and the V
    trace error of the plain FP32 path (|dV| below 0.1 mV for 90 % of
    neurons)."""
    x = inp.single_neurons(1024, seed=0)
    T, dt = 10_000, 0.01
    ref = oracle.simulate(inp.CLASSIC_HH, x["I"], x["V0"], T, dt, spk_cap=64)
    g = run_gpu(inp.CLASSIC_HH, x["I"], x["V0"], T, dt, hh.HH_PREC_POLY)
    assert g["status"] == 0
    assert np.array_equal(g["counts"], ref["counts"])
    errs = spike_time_errors(g, ref, dt)
    assert len(errs) == int((ref["counts"] > 0).sum())
    dV = np.abs(g["V"] - ref["V"]).max(0)
    print(f"poly: max|dV| median {np.median(dV):.2e} p90 {np.quantile(dV, 0.9):.2e} mV; "
          f"spike-time max {max(errs.values()):.2e} ms")
    assert max(errs.values()) <= T_TOL_MS
    assert np.quantile(dV, 0.9) < 0.1


def test_poly_multichannel_population():
    """Config 4 at 512 neurons over 500 ms: spike counts within +-1 for every
    neuron, spike times within 0.05 ms for >= 98 % of the matched neurons."""
    y = inp.multi_channel_neurons(512, seed=0)
    T, dt = 20_000, 0.025
    ref = oracle.simulate(inp.MULTI_CHANNEL, y["I"], y["V0"], T, dt, gbar=y["gbar"], trace=False,
                          spk_cap=128)
    g = run_gpu(inp.MULTI_CHANNEL, y["I"], y["V0"], T, dt, hh.HH_PREC_POLY, gbar=y["gbar"], trace=False)
    d = np.abs(g["counts"] - ref["counts"])
    errs = spike_time_errors(g, ref, dt)
    within = np.mean([e <= T_TOL_MS for e in errs.values()])
    print(f"poly multichannel: counts equal {(d == 0).mean():.4f}, max diff {d.max()}, "
          f"spike times within 0.05 ms {within:.4f}")
    assert d.max() <= 1
    assert within >= 0.98
    assert (ref["counts"] > 0).sum() > 100


def test_poly_multichannel_full_size_sampled():
    """The full 1e6 multi-channel population over 500 ms on the polynomial
    path; 256 sampled neurons re-simulated by the oracle: counts within +-1,
    identical for >= 95 %."""
    torch = _torch()
    y = inp.multi_channel_neurons(1_000_000, seed=0)
    T, dt, N = 20_000, 0.025, 1_000_000
    net = hh.Network(y["V0"], dt, I_const=y["I"], precision=hh.HH_PREC_POLY)
    net.set_channels(0, inp.MULTI_CHANNEL, gbar=y["gbar"])
    rec, b = hh.make_record(N, T, spike_cap=0)
    net.step(T, rec=rec)
    torch.cuda.synchronize()
    counts = b["counts"].cpu().numpy()
    assert int(net.readout(hh.HH_READ_STATUS)[0]) == 0
    net.close()
    idx = np.random.default_rng(2).choice(N, 256, replace=False)
    ref = oracle.simulate(inp.MULTI_CHANNEL, y["I"][idx], y["V0"][idx], T, dt,
                          gbar=y["gbar"][:, idx], trace=False, spk_cap=4)
    d = np.abs(counts[idx] - ref["counts"])
    assert d.max() <= 1
    assert (d == 0).mean() >= 0.95


def test_poly_fallback_outside_range():
    """Neurons held below the tabulated range (V0 = -130 .. -121 mV with a
    hyperpolarising current) and others inside it share warps: every warp
    with a lane outside takes the SFU arithmetic for that step: the lanes
    outside give the FAST path's bits, and every trace follows the oracle
    within the FAST path's own error over 5 ms."""
    N = 64
    V0 = np.where(np.arange(N) % 3 == 0, np.linspace(-130.0, -121.0, N), -65.0).astype(np.float32)
    I = np.where(np.arange(N) % 3 == 0, -40.0, np.linspace(0.0, 15.0, N)).astype(np.float32)
    T, dt = 500, 0.01
    ref = oracle.simulate(inp.CLASSIC_HH, I, V0, T, dt)
    assert (ref["V"][:, ::3] < hh.HH_POLY_V_LO).all()
    g = run_gpu(inp.CLASSIC_HH, I, V0, T, dt, hh.HH_PREC_POLY)
    f = run_gpu(inp.CLASSIC_HH, I, V0, T, dt, hh.HH_PREC_FAST)
    assert np.array_equal(g["V"][:, ::3], f["V"][:, ::3])  # the same SFU steps
    err_g, err_f = np.abs(g["V"] - ref["V"]).max(), np.abs(f["V"] - ref["V"]).max()
    print(f"poly fallback: max |dV| {err_g:.2e} mV (FAST {err_f:.2e})")
    assert err_g <= max(2.0 * err_f, 1e-3) and err_g <= 1e-2
