"""Closed-loop parity of the 38,000-neuron network over 1,000 ms (a script,
not collected by pytest: the FP64 oracle takes a minute or two on a
many-core host).

The GPU runs the benchmark network (in-degree 2,632, 1.0e8 synapses,
background, dt 0.025 ms, 40,000 steps) in FAST precision; the oracle runs
the same graph, background draws and initial state in FP64.  FP32 and FP64
trajectories of a recurrent spiking network separate in the end (chaos), so
the script reports how the agreement evolves: per-neuron spike counts equal
and within +-1 after 10 ms .. 1,000 ms, total spikes, and the population
rate in 1 ms bins (correlation, mean, spread, share of spikes in the top
1 % of 0.5 ms windows).

    python tests/parity_network_1s.py        # on a machine with the GPU
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2601_21407_gb300 import hh, inputs as inp  # noqa: E402


def main():
    import torch
    W = bench.W
    N, T = W["n"], bench.STEPS_PER_SIM
    g = inp.network(n=N, k_in=W["k_in"], exc_frac=W["exc_frac"], seed=W["seed"], mu=W["mu"],
                    sigma=W["sigma"])
    net = hh.Network(g["V0"], W["dt"], csr=(g["row_ptr"], g["col"], g["w"]), inh=g["inh"], syn=bench.SYN,
                     delay_steps=bench.DELAY, bg=bench.BG, seed=W["seed"], precision=hh.HH_PREC_FAST)
    net.set_channels(0, inp.CLASSIC_HH)
    rec, b = hh.make_record(N, T, spike_cap=4_000_000)
    net.step(T, rec=rec)
    torch.cuda.synchronize()
    status = int(net.readout(hh.HH_READ_STATUS)[0])
    steps_g, idx_g, _ = hh.spikes_to_numpy(b)
    cg = b["counts"].cpu().numpy().astype(np.int64)
    net.close()

    ref = oracle.simulate_network(inp.CLASSIC_HH, g, T, W["dt"], bench.DELAY, bench.SYN, bg=bench.BG,
                                  seed=W["seed"], spk_cap=256)
    cr = ref["counts"].astype(np.int64)
    ss = ref["spk_step"]
    res = {"status": status, "spikes_gpu": int(cg.sum()), "spikes_oracle": int(cr.sum()),
           "oracle_spike_cap_exceeded": int((cr > ss.shape[1]).sum())}
    for t_ms in (10, 50, 100, 200, 500, 1000):
        s_end = int(round(t_ms / W["dt"]))
        d = np.abs(np.bincount(idx_g[steps_g < s_end], minlength=N) - ((ss >= 0) & (ss < s_end)).sum(1))
        res[f"counts_{t_ms}ms"] = {"equal": float((d == 0).mean()), "within_1": float((d <= 1).mean()),
                                   "max_diff": int(d.max())}
    bins = np.arange(0, T + 1, bench.DELAY)
    sv = ss[ss >= 0]
    pg = np.histogram(steps_g, bins)[0] / N / (bench.DELAY * W["dt"] * 1e-3)
    pr = np.histogram(sv, bins)[0] / N / (bench.DELAY * W["dt"] * 1e-3)
    win = np.arange(0, T + 1, bench.DELAY // 2)
    top = max(1, (len(win) - 1) // 100)
    res["population_rate_1ms"] = {
        "correlation": float(np.corrcoef(pg, pr)[0, 1]),
        "mean_hz": [float(pg.mean()), float(pr.mean())], "std_hz": [float(pg.std()), float(pr.std())],
        "top1pct_window_share": [float(np.sort(np.histogram(steps_g, win)[0])[::-1][:top].sum() / len(steps_g)),
                                 float(np.sort(np.histogram(sv, win)[0])[::-1][:top].sum() / len(sv))]}
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
