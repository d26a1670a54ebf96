"""Checkpoint / resume of a network's whole dynamic state (hh_save_state,
hh_load_state), launch shapes of the window schedule (hh_set_launch_shape)
and their autotuning (hh_autotune).

A network saved after a call and restored, into itself or into a fresh
network built from the same descriptor, continues bit for bit as the
original did: V, gates, rasters and counts.  The launch shape changes
only the speed (delivery is order independent), so every shape gives the
same bits, and autotuning leaves the network in the state it found."""
import numpy as np
import pytest

from paper_2601_21407_gb300 import hh, inputs as inp

pytestmark = pytest.mark.gpu

SYN = {"tau_E": 5.0, "tau_I": 10.0, "E_E": 0.0, "E_I": -80.0, "area_cm2": 2.0e-4}
BG = {"rate_hz": 5.0, "K": 500, "w": 1.5}


def _torch():
    import torch
    return torch


def _net(g, precision=hh.HH_PREC_FAST, D=40, seed=4, models=(inp.CLASSIC_HH,), model_id=None):
    net = hh.Network(g["V0"], 0.025, csr=(g["row_ptr"], g["col"], g["w"]), inh=g["inh"], syn=SYN,
                     delay_steps=D, bg=BG, seed=seed, precision=precision, model_id=model_id)
    for k, m in enumerate(models):
        net.set_channels(k, m)
    return net


def _run(net, N, T):
    torch = _torch()
    rec, b = hh.make_record(N, T, trace=8, spike_cap=400_000)
    net.step(T, rec=rec)
    torch.cuda.synchronize()
    s = hh.spikes_to_numpy(b)
    order = np.lexsort((s[1], s[0]))
    return {"V": net.readout(hh.HH_READ_V), "gates": net.readout(hh.HH_READ_GATES),
            "gsyn": net.readout(hh.HH_READ_G_SYN), "counts": b["counts"].cpu().numpy(),
            "trace": b["V_trace"].cpu().numpy(), "spk": (s[0][order], s[1][order], s[2][order]),
            "t": int(net.readout(hh.HH_READ_TIME)[0]), "status": int(net.readout(hh.HH_READ_STATUS)[0])}


def _same(a, b):
    for k in ("V", "gates", "gsyn", "counts", "trace"):
        assert np.array_equal(a[k], b[k]), k
    for j in range(3):
        assert np.array_equal(a["spk"][j], b["spk"][j])
    assert a["t"] == b["t"] and a["status"] == b["status"] == 0


@pytest.mark.parametrize("precision,D", [(hh.HH_PREC_FAST, 40), (hh.HH_PREC_COMPENSATED, 7),
                                         (hh.HH_PREC_ACCURATE, 1)])
def test_resume_from_saved_state_is_bit_identical(precision, D):
    torch = _torch()
    g = inp.network(n=2000, k_in=150, seed=11, mu=0.3)
    a = _net(g, precision, D)
    _run(a, 2000, 1333)                      # an odd length: spikes in flight
    img = a.save_state()                     # pageable host memory
    assert img.nbytes == a.state_size()
    dev = torch.zeros(a.state_size(), dtype=torch.uint8, device="cuda")
    a.save_state(dev)                        # device memory
    assert np.array_equal(dev.cpu().numpy(), img)
    ref = _run(a, 2000, 2000)
    assert ref["counts"].sum() > 50
    # into a fresh network built from the same descriptor
    b = _net(g, precision, D)
    b.load_state(img)
    _same(_run(b, 2000, 2000), ref)
    # back into the original (a rewind), from the device copy
    a.load_state(dev)
    _same(_run(a, 2000, 2000), ref)
    a.close()
    b.close()


def test_load_state_rejects_a_different_network():
    g = inp.network(n=2000, k_in=150, seed=11, mu=0.3)
    a = _net(g)
    img = a.save_state()
    h = inp.network(n=1500, k_in=150, seed=11, mu=0.3)
    b = _net(h)
    with pytest.raises(hh.HHError) as e:
        b.load_state(img)
    assert e.value.status == hh.HH_EINVAL and "does not fit" in str(e.value)
    c = _net(g, D=20)
    with pytest.raises(hh.HHError):
        c.load_state(img)
    bad = img.copy()
    bad[:8] = 0
    with pytest.raises(hh.HHError) as e:
        a.load_state(bad)
    assert "not a state image" in str(e.value)
    with pytest.raises(hh.HHError):
        a.save_state(np.zeros(img.nbytes - 1, dtype=np.uint8))
    for n in (a, b, c):
        n.close()


def test_launch_shapes_give_identical_bits():
    g = inp.network(n=3000, k_in=300, seed=5, mu=0.0)
    out = []
    for block, route in ((0, 0), (32, 152), (64, 608), (128, 304)):
        net = _net(g)
        net.set_launch_shape(block, route)
        out.append(_run(net, 3000, 900))
        net.close()
    assert out[0]["counts"].sum() > 100
    for o in out[1:]:
        _same(o, out[0])
    net = _net(g)
    with pytest.raises(hh.HHError):
        net.set_launch_shape(48, 0)
    with pytest.raises(hh.HHError):
        net.set_launch_shape(0, -1)
    net.close()


def test_autotune_restores_state_and_keeps_results():
    """Mixed models (two installed) and a mid-run start: after tuning, the
    network's state is the one it had, and the rest of the run equals the
    untuned network's bit for bit."""
    g = inp.network(n=4000, k_in=200, seed=6, mu=0.0)
    mid = (np.arange(4000) % 2).astype(np.uint8)
    models = (inp.CLASSIC_HH, inp.MULTI_CHANNEL)
    a = _net(g, models=models, model_id=mid)
    b = _net(g, models=models, model_id=mid)
    _run(a, 4000, 250)
    _run(b, 4000, 250)
    before = a.save_state()
    rep = a.autotune(trial_steps=200)
    assert len(rep["candidates"]) == 10 and 0 <= rep["best"] < 10
    assert rep["candidates"][0][:2] == (0, 0)
    assert all(ms > 0 for _, _, ms in rep["candidates"])
    best = rep["candidates"][rep["best"]][2]
    assert rep["best"] == 0 or best <= 0.97 * rep["candidates"][0][2]
    assert np.array_equal(a.save_state(), before)
    ra, rb = _run(a, 4000, 600), _run(b, 4000, 600)
    _same(ra, rb)
    assert ra["counts"].sum() > 100
    a.close()
    b.close()
