"""GPU checks of the pull routing of dense windows (hh_set_route_pull): a
window routed by the pull over the in-CSR leaves the same delay-line bits as
the push over the out-CSR, so whole runs are bit-identical whichever way
each window is routed -- small and full-size networks, thresholds that
pull only some windows, windows of 1, 3, 20 and 64 steps, neurons that fire twice inside
one window (their earlier spikes are pushed), the table interpreter -- and
a pulled closed loop matches the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2601_21407_gb300 import hh, inputs as inp

from test_gpu_network import SYN, make_net

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _run(g, T, pull, D=40, bg=None, seed=3, dt=0.025, I=None, kernels=hh.HH_KERNELS_SPECIALISED, trace=False,
         chunks=None):
    torch = _torch()
    N = g["V0"].size
    net = make_net(g, dt=dt, D=D, bg=bg, seed=seed, I=I, kernels=kernels)
    if pull is not None:
        net.set_route_pull(pull)
    rec, b = hh.make_record(N, T, trace=N if trace else 0, spike_cap=4_000_000)
    for c in (chunks or [T]):
        net.step(c, rec=rec)
    torch.cuda.synchronize()
    out = {"V": net.readout(hh.HH_READ_V), "spk": hh.spikes_to_numpy(b), "counts": b["counts"].cpu().numpy(),
           "status": int(net.readout(hh.HH_READ_STATUS)[0])}
    if trace:
        out["V_trace"] = b["V_trace"].cpu().numpy()
    net.close()
    return out


def _same(a, b):
    assert np.array_equal(a["V"], b["V"])
    assert np.array_equal(a["counts"], b["counts"])
    for k in range(3):
        assert np.array_equal(a["spk"][k], b["spk"][k])


@pytest.mark.parametrize("D,kernels", [(1, hh.HH_KERNELS_SPECIALISED), (7, hh.HH_KERNELS_SPECIALISED),
                                       (40, hh.HH_KERNELS_SPECIALISED), (40, hh.HH_KERNELS_TABLE)])
def test_pull_equals_push(D, kernels):
    """1,000 neurons, in-degree 100, background, 100 ms: every window
    pulled, none pulled (the default) and windows of 20 spikes or more
    pulled give the same bits."""
    g = inp.network(n=1000, k_in=100, seed=4, mu=0.5)
    bg = {"rate_hz": 5.0, "K": 500, "w": 1.5}
    T = 4000
    push = _run(g, T, None, D=D, bg=bg, kernels=kernels)
    pull = _run(g, T, 0, D=D, bg=bg, kernels=kernels, chunks=[7, 1500, 2493])
    some = _run(g, T, 20, D=D, bg=bg, kernels=kernels)
    assert push["status"] == pull["status"] == some["status"] == 0
    assert push["counts"].sum() > 1000
    _same(push, pull)
    _same(push, some)


def test_pulled_closed_loop_matches_oracle():
    """The 200 ms closed loop of the small network with every window pulled:
    spike counts within +-1 of the oracle for every neuron, V within 1e-2 mV
    over the first 10 ms."""
    g = inp.network(n=1000, k_in=100, seed=4, mu=0.5)
    bg = {"rate_hz": 5.0, "K": 500, "w": 1.5}
    T = 8000
    ref = oracle.simulate_network(inp.CLASSIC_HH, g, T, 0.025, 40, SYN, bg=bg, seed=9, trace_idx=np.arange(1000))
    r = _run(g, T, 0, bg=bg, seed=9, trace=True)
    assert ref["counts"].sum() > 1000
    assert np.abs(r["counts"] - ref["counts"]).max() <= 1
    assert np.abs(r["V_trace"][:400] - ref["V"][:400]).max() < 1e-2


def test_pull_with_two_spikes_per_window():
    """Windows of 64 steps (D = 128 at dt 0.2 ms: 12.8 ms) and driven neurons
    firing at 60-130 Hz, so that many fire twice inside a window; the pull
    delivers each neuron's last spike and pushes the earlier ones."""
    g = inp.network(n=600, k_in=60, seed=6, mu=0.0)
    I = np.random.default_rng(1).uniform(10.0, 100.0, 600).astype(np.float32)
    T = 3000
    push = _run(g, T, -1, D=128, dt=0.2, I=I)
    pull = _run(g, T, 0, D=128, dt=0.2, I=I)
    st, ix, _ = push["spk"]
    win = st // 64
    key = win.astype(np.int64) * 600 + ix
    _, per = np.unique(key, return_counts=True)
    assert per.max() >= 2 and (per >= 2).sum() > 20
    _same(push, pull)


def test_pull_full_size_network():
    """The benchmark network (38,000 neurons, 1.0e8 synapses, background),
    100 ms: every window pulled, none pulled and windows of 2,000 spikes or
    more pulled give the same bits."""
    g = inp.network(n=38_000, k_in=2_632, seed=0)
    bg = {"rate_hz": 5.0, "K": 2106, "w": 0.368}
    T = 4000
    push = _run(g, T, None, bg=bg, seed=0)
    pull = _run(g, T, 0, bg=bg, seed=0)
    some = _run(g, T, 2000, bg=bg, seed=0)
    assert push["counts"].sum() > 10_000
    _same(push, pull)
    _same(push, some)


def test_pull_unsupported_networks():
    """Networks above 65,536 neurons, or with windows above 64 steps, cannot
    pull: asking them to is refused, turning pull off is accepted."""
    big = inp.network(n=70_000, k_in=4, seed=1)
    net = make_net(big)
    with pytest.raises(hh.HHError) as e:
        net.set_route_pull(0)
    assert e.value.status == hh.HH_EUNSUPPORTED
    net.set_route_pull(-1)
    net.close()
    g = inp.network(n=200, k_in=20, seed=2)
    net = make_net(g, D=200)
    with pytest.raises(hh.HHError) as e:
        net.set_route_pull(100)
    assert e.value.status == hh.HH_EUNSUPPORTED
    net.close()
