"""GPU parity of the network path (delay line, CSR routing, exponential
synapses, Poisson background) against the FP64 oracle: routing bit-exact in
2^-32 nS fixed point (small graphs and the full 1e8-synapse graph),
background counts bit-exact, closed-loop spike counts, batched networks with
mixed neuron models, determinism and resume, and CSR validation."""
import numpy as np
import pytest

import oracle
from paper_2601_21407_gb300 import hh, inputs as inp

pytestmark = pytest.mark.gpu

SYN = {"tau_E": 5.0, "tau_I": 10.0, "E_E": 0.0, "E_I": -80.0, "area_cm2": 2.0e-4}


def _torch():
    import torch
    return torch


def make_net(g, dt=0.025, D=40, bg=None, seed=0, precision=hh.HH_PREC_FAST, models=(inp.CLASSIC_HH,),
             model_id=None, I=None, kernels=hh.HH_KERNELS_SPECIALISED, stream=None):
    net = hh.Network(g["V0"], dt, csr=(g["row_ptr"], g["col"], g["w"]), inh=g["inh"], syn=SYN,
                     delay_steps=D, bg=bg, seed=seed, precision=precision, model_id=model_id,
                     I_const=I, kernels=kernels, stream=stream)
    for k, m in enumerate(models):
        net.set_channels(k, m)
    return net


def route_gpu(net, N, st, ix, n_window):
    torch = _torch()
    sE = torch.zeros((n_window, N), dtype=torch.int64, device="cuda")
    sI = torch.zeros_like(sE)
    net.route_spikes(torch.as_tensor(st, device="cuda"), torch.as_tensor(ix, device="cuda"),
                     n_window, sE, sI)
    torch.cuda.synchronize()
    return sE.cpu().numpy(), sI.cpu().numpy()


def to_fixed(x):
    y = x * 2.0**32
    assert np.array_equal(y, np.round(y))
    return y.astype(np.int64)


@pytest.mark.parametrize("n,k,seed,D", [(64, 10, 0, 1), (500, 50, 1, 7), (2000, 200, 2, 40),
                                        (3001, 17, 3, 40)])
def test_routing_bit_exact(n, k, seed, D):
    """Open-loop routing of a seeded raster: per-step, per-target delivered
    conductance equals the oracle's sums exactly (2^-32 nS fixed point)."""
    g = inp.network(n=n, k_in=k, seed=seed)
    st, ix = inp.spike_raster(n, 25, max(1, n // 50), seed + 100)
    Tw = 25 + D + 3
    net = make_net(g, D=D)
    gE, gI = route_gpu(net, n, st, ix, Tw)
    rE, rI = oracle.route(n, Tw, D, g["row_ptr"], g["col"], g["w"], g["inh"], st, ix)
    assert np.array_equal(gE, to_fixed(rE))
    assert np.array_equal(gI, to_fixed(rI))
    net.close()


def test_routing_full_size_graph():
    """The 38,000-neuron, 1.0e8-synapse graph: a 40-step raster with 1% of
    the neurons spiking per step (4.0e7 synaptic events) routes bit-exactly."""
    g = inp.network(n=38_000, k_in=2_632, seed=0)
    st, ix = inp.spike_raster(38_000, 40, 380, 1)
    net = make_net(g, D=40)
    out_ptr = net.readout(hh.HH_READ_N_OUT)
    assert out_ptr[-1] == 38_000 * 2_632
    gE, gI = route_gpu(net, 38_000, st, ix, 80)
    rE, rI = oracle.route(38_000, 80, 40, g["row_ptr"], g["col"], g["w"], g["inh"], st, ix)
    assert np.array_equal(gE, to_fixed(rE))
    assert np.array_equal(gI, to_fixed(rI))
    net.close()


def test_out_degree_matches_transpose():
    g = inp.network(n=1000, k_in=30, seed=7)
    net = make_net(g)
    deg = np.diff(net.readout(hh.HH_READ_N_OUT))
    assert np.array_equal(deg, np.bincount(g["col"], minlength=1000))
    net.close()


def test_background_counts_bit_exact():
    """Poisson background counts drawn on the GPU (Philox-4x32-10 word
    (t>>2, i, 1, t>>34)[t&3], inverse CDF on the 2^32 grid) equal the
    oracle's for every neuron over 9 steps (reconstructed from g_E)."""
    N = 4096
    bg = {"rate_hz": 5.0, "K": 2106, "w": 0.5}
    net = hh.Network(np.full(N, -65.0, np.float32), 0.025, syn=SYN, bg=bg, seed=123)
    net.set_channels(0, inp.CLASSIC_HH)
    thr = oracle.poisson_table(oracle.background_lambda(2106, 5.0, 0.025))
    dec = np.float32(np.exp(-0.025 / 5.0))
    prev = np.zeros(N, np.float32)
    total = 0
    for t in range(9):
        net.step(1)
        gsyn = net.readout(hh.HH_READ_G_SYN)[:N]
        k = np.rint((gsyn / dec - prev) / np.float32(0.5)).astype(int)
        kr = np.array([oracle.poisson_sample(oracle.background_word(123, t, i), thr) for i in range(N)])
        assert np.array_equal(k, kr), t
        total += kr.sum()
        prev = gsyn
    assert total > 0
    net.close()


@pytest.mark.parametrize("kernels", [hh.HH_KERNELS_SPECIALISED, hh.HH_KERNELS_PERSISTENT, hh.HH_KERNELS_TABLE])
def test_background_counts_in_network_bit_exact(kernels):
    """The background of a network with synapses (delay line, routing and
    list machinery active, every kernel schedule): with zero synaptic
    weights, g_E after each step reveals every neuron's count, and it equals
    the oracle's draw for every neuron and step."""
    N = 4096
    rng = np.random.default_rng(5)
    csr = (np.arange(0, 4 * N + 1, 4, dtype=np.int64), rng.integers(0, N, 4 * N).astype(np.int32),
           np.zeros(4 * N, np.float32))
    bg = {"rate_hz": 5.0, "K": 2106, "w": 0.5}
    net = hh.Network(np.full(N, -65.0, np.float32), 0.025, csr=csr, inh=np.zeros(N, np.uint8), syn=SYN,
                     delay_steps=6, bg=bg, seed=321, kernels=kernels)
    net.set_channels(0, inp.CLASSIC_HH)
    thr = oracle.poisson_table(oracle.background_lambda(2106, 5.0, 0.025))
    dec = np.float32(np.exp(-0.025 / 5.0))
    prev = np.zeros(N, np.float32)
    total = 0
    for t in range(9):
        net.step(1)
        gsyn = net.readout(hh.HH_READ_G_SYN)[:N]
        k = np.rint((gsyn / dec - prev) / np.float32(0.5)).astype(int)
        kr = np.array([oracle.poisson_sample(oracle.background_word(321, t, i), thr) for i in range(N)])
        assert np.array_equal(k, kr), t
        total += kr.sum()
        prev = gsyn
    assert total > 0
    net.close()


@pytest.mark.parametrize("prec,kernels", [(hh.HH_PREC_FAST, hh.HH_KERNELS_SPECIALISED),
                                          (hh.HH_PREC_ACCURATE, hh.HH_KERNELS_SPECIALISED),
                                          (hh.HH_PREC_COMPENSATED, hh.HH_KERNELS_SPECIALISED),
                                          (hh.HH_PREC_FAST, hh.HH_KERNELS_PERSISTENT),
                                          (hh.HH_PREC_FAST, hh.HH_KERNELS_TABLE),
                                          (hh.HH_PREC_POLY, hh.HH_KERNELS_SPECIALISED),
                                          (hh.HH_PREC_POLY, hh.HH_KERNELS_PERSISTENT)])
def test_closed_loop_small_network(prec, kernels):
    """1,000 neurons, in-degree 100, background, 200 ms closed loop: every
    neuron's spike count within +-1 of the oracle, and the V traces agree to
    1e-2 mV for the first 10 ms (before FP32/FP64 chaos separates them)."""
    torch = _torch()
    g = inp.network(n=1000, k_in=100, seed=4, mu=0.5)
    bg = {"rate_hz": 5.0, "K": 500, "w": 1.5}
    T = 8000
    ref = oracle.simulate_network(inp.CLASSIC_HH, g, T, 0.025, 40, SYN, bg=bg, seed=9,
                                  trace_idx=np.arange(1000))
    net = make_net(g, bg=bg, seed=9, precision=prec, kernels=kernels)
    rec, b = hh.make_record(1000, T, trace=1000, spike_cap=1_000_000)
    net.step(T, rec=rec)
    torch.cuda.synchronize()
    counts = b["counts"].cpu().numpy()
    assert ref["counts"].sum() > 1000
    assert np.abs(counts - ref["counts"]).max() <= 1
    V = b["V_trace"].cpu().numpy()
    assert np.abs(V[:400] - ref["V"][:400]).max() < 1e-2
    assert int(net.readout(hh.HH_READ_STATUS)[0]) == 0
    net.close()


@pytest.fixture(scope="module")
def network_38k_1s():
    """The benchmark network (38,000 neurons, in-degree 2,632, 1.0e8
    synapses, background, dt 0.025 ms) over 1,000 ms (40,000 steps) on the
    GPU in FAST precision and in the FP64 oracle on the same graph, initial
    state and background draws."""
    torch = _torch()
    g = inp.network(n=38_000, k_in=2_632, seed=0)
    bg = {"rate_hz": 5.0, "K": 2106, "w": 0.368}
    T = 40_000
    net = make_net(g, bg=bg, seed=0, precision=hh.HH_PREC_FAST)
    rec, b = hh.make_record(38_000, T, spike_cap=4_000_000)
    net.step(T, rec=rec)
    torch.cuda.synchronize()
    status = int(net.readout(hh.HH_READ_STATUS)[0])
    st, ix, _ = hh.spikes_to_numpy(b)
    n_stored = int(b["n_spikes"].item())
    net.close()
    ref = oracle.simulate_network(inp.CLASSIC_HH, g, T, 0.025, 40, SYN, bg=bg, seed=0, spk_cap=256)
    return {"T": T, "status": status, "n_spikes": n_stored, "gpu_step": st, "gpu_idx": ix,
            "ref_step": ref["spk_step"], "ref_counts": ref["counts"]}


def _counts_upto(r, t_ms, N=38_000):
    s_end = int(round(t_ms / 0.025))
    cg = np.bincount(r["gpu_idx"][r["gpu_step"] < s_end], minlength=N)
    ss = r["ref_step"]
    cr = ((ss >= 0) & (ss < s_end)).sum(1)
    return cg, cr


def test_network_full_size_first_10ms(network_38k_1s):
    """The full network against the oracle over its first 10 ms: spike
    counts identical for >= 99.9 % of neurons, totals within 0.1 %."""
    r = network_38k_1s
    cg, cr = _counts_upto(r, 10)
    assert (cg == cr).mean() >= 0.999
    assert abs(int(cg.sum()) - int(cr.sum())) <= 0.001 * cr.sum() + 2


def test_network_full_size_1000ms(network_38k_1s):
    """Closed-loop parity over the full 1,000 ms.  FP32 and FP64 trajectories
    of a recurrent spiking network separate in the end (chaos: which neurons
    drift, and when, changes with any change of the FP32 rounding), so the
    bar is stated per horizon: per-neuron spike counts within +-1 for every
    neuron up to 200 ms, for >= 99.99 % of neurons at 500 ms and >= 99.9 % at
    1,000 ms; total spikes within 0.1 %; the population rate in 1 ms bins
    correlated at >= 0.95 over the first 500 ms, and over the whole second
    the same mean within 1 % and spread within 10 % (the timing of the later
    bursts follows the realisation: its correlation over the second was
    0.84-0.98 across kernels differing only in rounding)."""
    r = network_38k_1s
    assert r["status"] == 0
    ref_cap = r["ref_step"].shape[1]
    assert (r["ref_counts"] <= ref_cap).all()
    assert r["n_spikes"] == len(r["gpu_idx"])
    stats = {}
    for t_ms in (50, 100, 200, 500, 1000):
        cg, cr = _counts_upto(r, t_ms)
        d = np.abs(cg - cr)
        stats[t_ms] = ((d == 0).mean(), (d <= 1).mean(), int(d.max()), int(cg.sum()), int(cr.sum()))
        print(f"{t_ms} ms: equal {stats[t_ms][0]:.5f}, within 1 {stats[t_ms][1]:.5f}, max {d.max()}, "
              f"spikes {cg.sum()} vs {cr.sum()}")
    bins = np.arange(0, r["T"] + 1, 40)
    sv = r["ref_step"][r["ref_step"] >= 0]
    pg = np.histogram(r["gpu_step"], bins)[0].astype(np.float64)
    pr = np.histogram(sv, bins)[0].astype(np.float64)
    corr = float(np.corrcoef(pg, pr)[0, 1])
    h = len(pg) // 2
    corr_half = float(np.corrcoef(pg[:h], pr[:h])[0, 1])
    print(f"population rate (1 ms bins): correlation {corr:.3f} (first 500 ms {corr_half:.3f}), "
          f"mean {pg.mean():.3f} vs {pr.mean():.3f}, std {pg.std():.2f} vs {pr.std():.2f} spikes/bin")
    for t_ms in (50, 100, 200):
        assert stats[t_ms][2] <= 1, (t_ms, stats[t_ms])
    assert stats[500][1] >= 0.9999, stats[500]
    assert stats[1000][1] >= 0.999, stats[1000]
    assert abs(stats[1000][3] - stats[1000][4]) <= 0.001 * stats[1000][4]
    assert corr_half >= 0.95
    assert abs(pg.mean() - pr.mean()) <= 0.01 * pr.mean()
    assert abs(pg.std() - pr.std()) <= 0.1 * pr.std()


def test_batched_networks_mixed_models():
    """Several independent networks (block-diagonal CSR) in one launch, with
    half of them classic HH and half multi-channel neurons: spike counts
    within +-1 of the oracle over 100 ms."""
    torch = _torch()
    bn = inp.batched_networks(n_nets=6, n_min=200, n_max=1500, k_min=20, k_max=80, seed=2)
    N = int(bn["offsets"][-1])
    bg = {"rate_hz": 5.0, "K": 600, "w": 1.2}
    T = 4000
    ref = oracle.simulate_network([inp.CLASSIC_HH, inp.MULTI_CHANNEL], bn, T, 0.025, 40, SYN, bg=bg,
                                  seed=3, model_id=bn["model_id"])
    net = make_net(bn, bg=bg, seed=3, models=(inp.CLASSIC_HH, inp.MULTI_CHANNEL),
                   model_id=bn["model_id"])
    rec, b = hh.make_record(N, T, spike_cap=2_000_000)
    net.step(T, rec=rec)
    torch.cuda.synchronize()
    counts = b["counts"].cpu().numpy()
    assert ref["counts"].sum() > 500
    d = np.abs(counts - ref["counts"])
    assert (d <= 1).mean() >= 0.99
    net.close()


def test_batched_networks_config5_shape():
    """Batched heterogeneous networks with the shape of the 64-network
    workload -- sizes log-uniform, in-degree uniform in 100..1,000, half the
    networks classic HH and half multi-channel, background 600 sources x 5 Hz
    x 1.2 nS, 200 ms -- scaled to 16 networks of 1,000-6,000 neurons so the
    oracle runs in seconds.  Closed-loop parity per horizon (as for the
    single large network: FP32 and FP64 trajectories of a chaotic network
    separate): counts within +-1 for every neuron at 50 ms, for >= 99.9 % at
    100 ms and >= 98 % at 200 ms; total spikes within 0.5 % and every
    network's total within 6 % (+3 spikes).  Measured: 100 %, 99.984 %,
    98.68 %; 240,964 vs 240,527 spikes; the twelve networks with in-degree
    above 400 end with exactly the oracle's totals, and the four sparsest
    (in-degree 139-293), whose activity is asynchronous, within 4.4 %."""
    torch = _torch()
    bn = inp.batched_networks(n_nets=16, n_min=1000, n_max=6000, k_min=100, k_max=1000, seed=7)
    N = int(bn["offsets"][-1])
    bg = {"rate_hz": 5.0, "K": 600, "w": 1.2}
    T = 8000
    models = [inp.CLASSIC_HH, inp.MULTI_CHANNEL]
    ref = oracle.simulate_network(models, bn, T, 0.025, 40, SYN, bg=bg, seed=3, model_id=bn["model_id"],
                                  spk_cap=128)
    net = make_net(bn, bg=bg, seed=3, models=tuple(models), model_id=bn["model_id"])
    rec, b = hh.make_record(N, T, spike_cap=4_000_000)
    net.step(T, rec=rec)
    torch.cuda.synchronize()
    assert int(net.readout(hh.HH_READ_STATUS)[0]) == 0
    st, ix, _ = hh.spikes_to_numpy(b)
    net.close()
    assert (ref["counts"] <= ref["spk_step"].shape[1]).all()
    off = bn["offsets"]
    stats = {}
    for t_ms in (50, 100, 200):
        s_end = int(round(t_ms / 0.025))
        cg = np.bincount(ix[st < s_end], minlength=N)
        ss = ref["spk_step"]
        cr = ((ss >= 0) & (ss < s_end)).sum(1)
        d = np.abs(cg - cr)
        per_net = [(int(cg[off[k]:off[k + 1]].sum()), int(cr[off[k]:off[k + 1]].sum())) for k in range(16)]
        stats[t_ms] = ((d == 0).mean(), (d <= 1).mean(), int(d.max()), int(cg.sum()), int(cr.sum()), per_net)
        print(f"{t_ms} ms: equal {stats[t_ms][0]:.5f}, within 1 {stats[t_ms][1]:.5f}, max {d.max()}, "
              f"spikes {cg.sum()} vs {cr.sum()}")
    print("N", N, "synapses", bn["col"].size, "per-network totals at 200 ms", stats[200][5])
    assert stats[200][4] > 5000
    assert stats[50][2] <= 1
    assert stats[100][1] >= 0.999
    assert stats[200][1] >= 0.98
    assert abs(stats[200][3] - stats[200][4]) <= 0.005 * stats[200][4]
    for g_tot, r_tot in stats[200][5]:
        assert abs(g_tot - r_tot) <= 0.06 * r_tot + 3


def test_deterministic_and_resumable():
    """Two runs from the same state give bit-identical rasters (fixed-point
    delivery is order independent), splitting a run across calls at points
    that do not align with the delay windows changes no bit, and the
    single-launch persistent schedule equals the launch-per-window one."""
    torch = _torch()
    g = inp.network(n=3000, k_in=300, seed=5, mu=0.0)
    bg = {"rate_hz": 5.0, "K": 500, "w": 1.5}

    def run(chunks, kernels=hh.HH_KERNELS_SPECIALISED):
        net = make_net(g, bg=bg, seed=1, kernels=kernels)
        rec, b = hh.make_record(3000, sum(chunks), spike_cap=500_000)
        for c in chunks:
            net.step(c, rec=rec)
        torch.cuda.synchronize()
        v = net.readout(hh.HH_READ_V)
        s = hh.spikes_to_numpy(b)
        assert int(net.readout(hh.HH_READ_STATUS)[0]) == 0
        net.close()
        return v, s

    a = run([2000])
    b = run([2000])
    c = run([13, 401, 999, 587])
    d = run([2000], hh.HH_KERNELS_PERSISTENT)
    e = run([13, 401, 999, 587], hh.HH_KERNELS_PERSISTENT)
    for x in (b, c, d, e):
        assert np.array_equal(a[0], x[0])
        for k in range(3):
            assert np.array_equal(a[1][k], x[1][k])
    assert len(a[1][0]) > 100


@pytest.mark.parametrize("D,chunks", [(2, [1, 300, 99]), (7, [400]), (13, [5, 6, 389]), (40, [1000])])
def test_persistent_matches_launches(D, chunks):
    """The single cooperative launch (windows of D/2 steps, routing warps
    delivering the previous window while the neuron threads integrate the
    next) gives bit-identical V and rasters to one launch per window, for
    odd and minimal delays and calls of any length."""
    torch = _torch()
    g = inp.network(n=2000, k_in=150, seed=11, mu=0.3)
    bg = {"rate_hz": 5.0, "K": 500, "w": 1.5}
    out = []
    for kernels in (hh.HH_KERNELS_PERSISTENT, hh.HH_KERNELS_SPECIALISED):
        net = make_net(g, D=D, bg=bg, seed=4, kernels=kernels)
        net.profile(True)
        rec, b = hh.make_record(2000, sum(chunks), trace=16, spike_cap=400_000)
        for c in chunks:
            net.step(c, rec=rec)
        torch.cuda.synchronize()
        kt = net.kernel_times()
        out.append((net.readout(hh.HH_READ_V), hh.spikes_to_numpy(b), b["V_trace"].cpu().numpy(),
                    int(net.readout(hh.HH_READ_STATUS)[0]), kt))
        net.close()
    (va, sa, ta, sta, kta), (vb, sb, tb, stb, ktb) = out
    assert sta == 0 and stb == 0
    assert kta["neuron"][0] == len(chunks) and kta["route"][0] == 0
    assert np.array_equal(va, vb) and np.array_equal(ta, tb)
    for k in range(3):
        assert np.array_equal(sa[k], sb[k])
    assert len(sa[0]) > 50


def test_persistent_wait_expiry_reports_status():
    """The persistent kernel's bounded waits on other blocks' progress, made to
    run out: with the progress bound at 0 ns every waiter gives up at once,
    records HH_STATUS_BARRIER_TIMEOUT and returns, so the call ends instead of
    hanging; with the default bound restored, a reset and the same run match
    the launch-per-window schedule bit for bit."""
    torch = _torch()
    g = inp.network(n=2000, k_in=150, seed=11, mu=0.3)
    bg = {"rate_hz": 5.0, "K": 500, "w": 1.5}
    T = 400
    net = make_net(g, D=40, bg=bg, seed=4, kernels=hh.HH_KERNELS_PERSISTENT)
    rec, b = hh.make_record(2000, T, spike_cap=400_000)
    try:
        hh.hh_set_wait_limits(progress_ns=0)
        net.step(T, rec=rec)
        torch.cuda.synchronize()
    finally:
        hh.hh_set_wait_limits()
    assert int(net.readout(hh.HH_READ_STATUS)[0]) & hh.HH_STATUS_BARRIER_TIMEOUT
    net.reset()
    b["counts"].zero_()
    net.step(T, rec=rec)
    torch.cuda.synchronize()
    assert int(net.readout(hh.HH_READ_STATUS)[0]) == 0
    va, ca = net.readout(hh.HH_READ_V), b["counts"].cpu().numpy()
    net.close()
    net = make_net(g, D=40, bg=bg, seed=4, kernels=hh.HH_KERNELS_SPECIALISED)
    rec2, b2 = hh.make_record(2000, T, spike_cap=400_000)
    net.step(T, rec=rec2)
    torch.cuda.synchronize()
    assert np.array_equal(va, net.readout(hh.HH_READ_V))
    assert np.array_equal(ca, b2["counts"].cpu().numpy()) and ca.sum() > 0
    net.close()


@pytest.mark.parametrize("kernels", [hh.HH_KERNELS_SPECIALISED, hh.HH_KERNELS_TABLE])
def test_graph_schedule_matches_stream_schedule(kernels):
    """On a caller stream the window schedule of each call is captured into
    a CUDA graph (executables reused when a call has the same shape); with
    profiling on it is enqueued launch by launch.  Both give bit-identical V,
    rasters and traces over calls of repeated and changing lengths."""
    torch = _torch()
    g = inp.network(n=3000, k_in=300, seed=5, mu=0.0)
    bg = {"rate_hz": 5.0, "K": 500, "w": 1.5}
    chunks = [400, 400, 400, 13, 400, 787, 400]
    s = torch.cuda.Stream()

    def run(profile):
        net = make_net(g, bg=bg, seed=1, kernels=kernels, stream=s.cuda_stream)
        net.profile(profile)
        rec, b = hh.make_record(3000, max(chunks), trace=8, spike_cap=500_000)
        traces = []
        for c in chunks:
            net.step(c, rec=rec)
            s.synchronize()
            traces.append(b["V_trace"][:c].cpu().numpy().copy())
        s.synchronize()
        out = (net.readout(hh.HH_READ_V), hh.spikes_to_numpy(b), traces,
               int(net.readout(hh.HH_READ_STATUS)[0]))
        net.close()
        return out

    a, p = run(False), run(True)
    assert a[3] == 0 and p[3] == 0
    assert np.array_equal(a[0], p[0])
    for k in range(3):
        assert np.array_equal(a[1][k], p[1][k])
    for x, y in zip(a[2], p[2]):
        assert np.array_equal(x, y)
    assert len(a[1][0]) > 100


def test_repeated_call_relaunches_same_schedule():
    """A call identical to the previous one (same state after a reset, same
    arguments) relaunches the captured schedule; a call that differs only in
    its record buffers or its length is captured anew and writes where it
    is told."""
    torch = _torch()
    g = inp.network(n=3000, k_in=300, seed=5, mu=0.0)
    bg = {"rate_hz": 5.0, "K": 500, "w": 1.5}
    s = torch.cuda.Stream()
    net = make_net(g, bg=bg, seed=1, stream=s.cuda_stream)
    V0 = torch.as_tensor(g["V0"], device="cuda")
    recs = [hh.make_record(3000, 600, trace=4, spike_cap=200_000) for _ in range(2)]

    def run(k, n):
        rec, b = recs[k]
        with torch.cuda.stream(s):
            b["counts"].zero_()
            b["n_spikes"].zero_()
            b["V_trace"].zero_()
        net.reset(V0)
        net.step(n, rec=rec)
        s.synchronize()
        return (net.readout(hh.HH_READ_V), b["counts"].cpu().numpy().copy(), b["V_trace"][:n].cpu().numpy().copy())

    a = run(0, 600)
    b = run(0, 600)
    with torch.cuda.stream(s):
        recs[0][1]["counts"].fill_(-7)
    c = run(1, 600)
    assert (recs[0][1]["counts"].cpu().numpy() == -7).all()
    d = run(1, 450)
    e = run(1, 600)
    assert a[1].sum() > 100
    for x in (b, c, e):
        assert np.array_equal(a[0], x[0]) and np.array_equal(a[1], x[1]) and np.array_equal(a[2], x[2])
    assert np.array_equal(a[2][:450], d[2])
    assert int(net.readout(hh.HH_READ_STATUS)[0]) == 0
    net.close()


def test_reset_restores_initial_state():
    torch = _torch()
    g = inp.network(n=800, k_in=80, seed=6, mu=0.5)
    bg = {"rate_hz": 5.0, "K": 500, "w": 1.5}
    net = make_net(g, bg=bg, seed=2)
    out = []
    for _ in range(2):
        rec, b = hh.make_record(800, 1000, spike_cap=100_000)
        net.reset()
        net.step(1000, rec=rec)
        torch.cuda.synchronize()
        out.append(hh.spikes_to_numpy(b))
    assert all(np.array_equal(out[0][k], out[1][k]) for k in range(3))
    assert int(net.readout(hh.HH_READ_TIME)[0]) == 1000
    net.close()


@pytest.mark.parametrize("what", ["col", "weight_neg", "weight_nan", "row_ptr"])
def test_invalid_csr_rejected(what):
    g = inp.network(n=100, k_in=10, seed=0)
    col, w, rp = g["col"].copy(), g["w"].copy(), g["row_ptr"].copy()
    if what == "col":
        col[17] = 100
    elif what == "weight_neg":
        w[3] = -0.5
    elif what == "weight_nan":
        w[5] = np.nan
    else:
        rp[50] = rp[49] - 1
    with pytest.raises(hh.HHError) as e:
        hh.Network(g["V0"], 0.025, csr=(rp, col, w), inh=g["inh"], syn=SYN, delay_steps=40)
    assert e.value.status == hh.HH_EINVAL


def test_profile_counts_launches():
    """D = 40: windows of D/2 steps, so 400 steps are 20 neuron and 20
    routing launches (routing overlaps the next window on a second stream);
    the persistent mode makes it one cooperative launch per call; D = 1
    keeps one launch pair per step."""
    g = inp.network(n=500, k_in=20, seed=8)
    bg = {"rate_hz": 5.0, "K": 500, "w": 1.0}
    net = make_net(g, bg=bg)
    net.profile(True)
    net.step(400)
    kt = net.kernel_times()
    net.profile(False)
    assert kt["neuron"][0] == 20 and kt["route"][0] == 20
    assert kt["neuron"][1] > 0
    net.close()
    net = make_net(g, bg=bg, kernels=hh.HH_KERNELS_PERSISTENT)
    net.profile(True)
    net.step(400)
    kt = net.kernel_times()
    assert kt["neuron"][0] == 1 and kt["route"][0] == 0
    net.close()
    net = make_net(g, D=1)
    net.profile(True)
    net.step(30)
    kt = net.kernel_times()
    assert kt["neuron"][0] == 30 and kt["route"][0] == 30
    net.close()
