"""The learned multi-step surrogate (hh_surrogate_train / hh_surrogate_enable
via the C ABI): training converges on windows from the plain integrator,
windows outside the trained envelope are integrated by the plain kernel
(with every window declined the run is bit-identical to the plain path), and
the error against the plain path and the FP64 oracle is measured and
reported.  The MLP learns the correction to one exponential-Euler step over
the whole window.  Without its per-neuron error estimate the surrogate
misses the spike-time part of the accuracy target (spike counts within +-1
and spike times within 0.05 ms for every neuron); with a tight estimate it
meets it on about half of the windows.  The tests record the achieved
figures."""
import json

import numpy as np
import pytest

import oracle
from paper_2601_21407_gb300 import hh, inputs as inp

pytestmark = pytest.mark.gpu

DT = 0.025


def _torch():
    import torch
    return torch


def run(y, T, *, surrogate=None, precision=hh.HH_PREC_FAST):
    torch = _torch()
    N = y["V0"].size
    net = hh.Network(y["V0"], DT, I_const=y["I"], precision=precision)
    net.set_channels(0, inp.MULTI_CHANNEL, gbar=y["gbar"])
    rep = None
    if surrogate is not None:
        rep = net.train_surrogate(**surrogate)
        net.enable_surrogate(True)
    rec, b = hh.make_record(N, T, spike_cap=50 * N + 1000)
    net.step(T, rec=rec)
    torch.cuda.synchronize()
    out = {"counts": b["counts"].cpu().numpy(), "spk": hh.spikes_to_numpy(b), "rep": rep,
           "V": net.readout(hh.HH_READ_V), "status": int(net.readout(hh.HH_READ_STATUS)[0])}
    if surrogate is not None:
        out["stats"] = net.surrogate_stats()
    net.close()
    return out


SMALL_TRAIN = dict(train_neurons=4096, train_windows=200_000, epochs=60, batch=2048)


def test_training_converges():
    """Held-out mean squared error of the scaled 10-step increments falls
    below 1 % of their variance."""
    y = inp.multi_channel_neurons(2048, seed=5)
    r = run(y, 40, surrogate=dict(v_envelope=-55.0, **SMALL_TRAIN))
    rep = r["rep"]
    assert rep["train_windows"] == 200_000
    assert rep["val_loss"] < 0.01, rep
    assert rep["out_scale_V"] > 0


def test_declined_windows_reproduce_plain_path():
    """Neurons driven by a current far outside the trained range (I = 200
    uA/cm^2 against training currents in [0, 15]) fail the feature envelope in
    every window, so every window goes through the decline list to the plain
    kernel: V, spike counts and rasters are bit-identical to the plain path
    and no window is counted as accepted."""
    y = inp.multi_channel_neurons(3000, seed=6)
    y = dict(y)
    y["I"] = np.full(3000, 200.0, np.float32)
    T = 4003  # 400 whole windows + 3 plain steps
    p = run(y, T)
    s = run(y, T, surrogate=dict(v_envelope=-55.0, **SMALL_TRAIN))
    assert s["stats"][0] == 0 and s["stats"][1] == 3000 * 400
    assert np.array_equal(p["V"], s["V"])
    assert np.array_equal(p["counts"], s["counts"])
    for k in range(3):
        assert np.array_equal(p["spk"][k], s["spk"][k])
    assert p["counts"].sum() > 0


def test_untrainable_envelope_is_rejected():
    """An envelope that no training window stays below is an error."""
    y = inp.multi_channel_neurons(256, seed=8)
    net = hh.Network(y["V0"], DT, I_const=y["I"], precision=hh.HH_PREC_FAST)
    net.set_channels(0, inp.MULTI_CHANNEL, gbar=y["gbar"])
    with pytest.raises(hh.HHError) as e:
        net.train_surrogate(v_envelope=-200.0, **SMALL_TRAIN)
    assert e.value.status == hh.HH_EINVAL
    net.close()


def _spike_time_agreement(a, b, N, tol_ms=0.05):
    """Share of neurons with equal counts in the two runs whose spike times
    all agree within tol_ms, over the neurons with equal counts."""
    sa, ia, fa = a["spk"]
    sb, ib, fb = b["spk"]
    ta = (sa + fa) * DT
    tb = (sb + fb) * DT
    oa, ob = np.argsort(ia, kind="stable"), np.argsort(ib, kind="stable")
    ca, cb = np.bincount(ia, minlength=N), np.bincount(ib, minlength=N)
    pa, pb = np.concatenate([[0], np.cumsum(ca)]), np.concatenate([[0], np.cumsum(cb)])
    eq = np.nonzero(ca == cb)[0]
    ok = 0
    for i in eq:
        x, y = np.sort(ta[oa[pa[i]:pa[i + 1]]]), np.sort(tb[ob[pb[i]:pb[i + 1]]])
        ok += x.size == 0 or np.abs(x - y).max() <= tol_ms
    return ok / max(1, eq.size)


def test_surrogate_error_is_measured():
    """Surrogate run of 4,096 multi-channel neurons for 500 ms without the
    error estimate: the share of neuron-windows taken from the MLP and the
    spike-count and spike-time errors against the plain FP32 path and the
    FP64 oracle, asserted at the levels this surrogate reaches (measured: 85 %
    of windows accepted, counts within +-1 of the plain path for 99.0-99.2 %
    of neurons and of the oracle for 99.6 %, spike times within 0.05 ms for
    62-64 % of the count-equal neurons).  The +-1 / 0.05 ms target is not met
    without the estimate; the plain path itself meets it against the
    oracle."""
    y = inp.multi_channel_neurons(4096, seed=7)
    T = 20_000
    plain = run(y, T)
    sur = run(y, T, surrogate=dict(v_envelope=-55.0, train_neurons=16384, train_windows=1_000_000,
                                   epochs=30, batch=8192))
    acc, dec = sur["stats"]
    assert sur["status"] == 0
    assert acc / (acc + dec) > 0.3
    assert np.isfinite(sur["V"]).all()
    dc = np.abs(sur["counts"] - plain["counts"])
    idx = np.random.default_rng(0).choice(4096, 256, replace=False)
    ref = oracle.simulate(inp.MULTI_CHANNEL, y["I"][idx], y["V0"][idx], T, DT, gbar=y["gbar"][:, idx],
                          trace=False, spk_cap=4)
    dco = np.abs(sur["counts"][idx] - ref["counts"])
    report = {"accepted_frac": acc / (acc + dec), "count_within_1_vs_plain": float((dc <= 1).mean()),
              "count_equal_vs_plain": float((dc == 0).mean()),
              "count_within_1_vs_oracle": float((dco <= 1).mean()),
              "plain_count_within_1_vs_oracle": float(
                  (np.abs(plain["counts"][idx] - ref["counts"]) <= 1).mean()),
              "val_loss": sur["rep"]["val_loss"],
              "spike_times_within_0.05ms_of_plain": _spike_time_agreement(sur, plain, 4096)}
    print(json.dumps(report))
    # the plain path itself meets the count target against the oracle
    assert report["plain_count_within_1_vs_oracle"] == 1.0
    # the levels the surrogate reaches
    assert report["accepted_frac"] >= 0.75
    assert report["count_within_1_vs_plain"] >= 0.97
    assert report["count_within_1_vs_oracle"] >= 0.97
    assert report["spike_times_within_0.05ms_of_plain"] >= 0.5


def test_error_estimate_controls_accuracy():
    """The per-neuron error estimate (the size of the MLP's correction to one
    exponential-Euler step over the whole window, hh_surrogate_desc.err_V /
    err_p) hands every window that needs a larger correction to the plain
    kernel.  Tightening it trades accepted windows for accuracy (4,096
    multi-channel neurons, 500 ms; measured: at 0.1 mV / 0.004, 79 % of
    windows accepted and counts within +-1 of the plain path for 99.0-99.1 %
    of neurons; at 0.01 mV / 0.0005, 54 % accepted, every neuron's count
    equal to the plain path's and spike times within 0.05 ms for 99.7-99.8 %
    of them -- the accuracy target).  The training windows are appended by
    atomics, so their order, and the trained weights, vary slightly from run
    to run: the bars sit below the measured levels."""
    y = inp.multi_channel_neurons(4096, seed=7)
    T = 20_000
    plain = run(y, T)
    idx = np.random.default_rng(0).choice(4096, 256, replace=False)
    ref = oracle.simulate(inp.MULTI_CHANNEL, y["I"][idx], y["V0"][idx], T, DT, gbar=y["gbar"][:, idx],
                          trace=False, spk_cap=4)
    base = dict(v_envelope=-55.0, train_neurons=16384, train_windows=1_000_000, epochs=30, batch=8192)
    out = {}
    for key, (eV, ep) in {"mid": (0.1, 0.004), "tight": (0.01, 0.0005)}.items():
        sur = run(y, T, surrogate=dict(base, err_V=eV, err_p=ep))
        acc, dec = sur["stats"]
        dc = np.abs(sur["counts"] - plain["counts"])
        out[key] = {"accepted_frac": acc / (acc + dec), "within_1": float((dc <= 1).mean()),
                    "max_diff": int(dc.max()),
                    "within_1_oracle": float((np.abs(sur["counts"][idx] - ref["counts"]) <= 1).mean()),
                    "times": _spike_time_agreement(sur, plain, 4096)}
        assert sur["status"] == 0
    print(json.dumps(out))
    assert out["mid"]["accepted_frac"] >= 0.6 and out["mid"]["within_1"] >= 0.97
    assert out["tight"]["accepted_frac"] >= 0.4
    assert out["tight"]["within_1"] >= 0.999 and out["tight"]["within_1_oracle"] >= 0.99
    assert out["tight"]["times"] >= 0.98
    # looser tolerance, more windows from the MLP
    assert out["mid"]["accepted_frac"] > out["tight"]["accepted_frac"]


def test_error_estimate_tolerances_are_checked():
    y = inp.multi_channel_neurons(256, seed=8)
    net = hh.Network(y["V0"], DT, I_const=y["I"], precision=hh.HH_PREC_FAST)
    net.set_channels(0, inp.MULTI_CHANNEL, gbar=y["gbar"])
    for eV, ep in ((-1.0, 0.01), (0.1, 0.0), (float("nan"), 0.01)):
        with pytest.raises(hh.HHError) as e:
            net.train_surrogate(v_envelope=-55.0, err_V=eV, err_p=ep, **SMALL_TRAIN)
        assert e.value.status == hh.HH_EINVAL
    net.close()
