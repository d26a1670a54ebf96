#!/usr/bin/env python
"""Benchmark of the HH hot path on the sparse conductance-based network.

Workload (synthetic, seeded): 38,000 classic HH neurons (80% excitatory),
fixed in-degree 2,632 with uniformly random sources (1.0e8 synapses, CSR),
lognormal weights (mu=-1, sigma=0.5 nS), exponential synapses (tau_E 5 ms,
tau_I 10 ms, E_E 0, E_I -80 mV), 1 ms delay, Poisson background, dt 0.025 ms,
1,000 ms of simulated time per step (40,000 time steps).

One bench step = reset the network state and simulate the full 1,000 ms:
every time step runs delivery from the delay line, the background draw, the
rates/gates/V update, threshold detection, spike compaction, routing over the
CSR graph and synaptic decay.  value = neuron-steps/s over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2601_21407_gb300 import inputs as inp  # noqa: E402

W = dict(n=38_000, k_in=2_632, exc_frac=0.8, mu=-1.0, sigma=0.5, tau_E=5.0, tau_I=10.0,
         E_E=0.0, E_I=-80.0, area_cm2=2.0e-4, delay_ms=1.0, dt=0.025, T_ms=1000.0,
         bg_rate_hz=5.0, bg_K=2_106, bg_w_nS=0.368, seed=0)
STEPS_PER_SIM = int(round(W["T_ms"] / W["dt"]))
DELAY = int(round(W["delay_ms"] / W["dt"]))
SYN = {"tau_E": W["tau_E"], "tau_I": W["tau_I"], "E_E": W["E_E"], "E_I": W["E_I"],
       "area_cm2": W["area_cm2"]}
BG = {"rate_hz": W["bg_rate_hz"], "K": W["bg_K"], "w": W["bg_w_nS"]}
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes (read + write) of one 20-step window launch of the 38k network
# (ncu, cold L2; the current window kernel)
WINDOW_TRAFFIC_BYTES = 14_508_544
# SFU (MUFU) issue rate per SM per clock for ex2/rcp on this architecture and
# the SM count / maximum clock of the part.
SM_COUNT, MUFU_PER_SM_CLK, FP32_PER_SM_CLK = 152, 16, 128


def workload_config():
    return {"workload": "hh_sparse_network_38k",
            "neurons": W["n"], "in_degree": W["k_in"], "synapses": W["n"] * W["k_in"],
            "exc_frac": W["exc_frac"], "weights": "lognormal(mu=-1,sigma=0.5) nS",
            "tau_E_ms": W["tau_E"], "tau_I_ms": W["tau_I"], "delay_ms": W["delay_ms"],
            "dt_ms": W["dt"], "sim_ms": W["T_ms"],
            "background": f"{W['bg_K']} Poisson sources x {W['bg_rate_hz']} Hz x {W['bg_w_nS']} nS",
            "model": "classic squid-axon HH (Na, K, leak)", "precision_mode": "fast",
            "l2": "inputs larger than L2 (CSR 800 MB vs 129 MB L2)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler is producing rows; the
            # rows written before it are not counted
            t_end = time.time() + 3.0
            self.skip = 0
            while time.time() < t_end:
                with open(self.path) as f:
                    self.skip = sum(1 for _ in f)
                if self.skip > 0 or self.proc.poll() is not None:
                    break
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                try:
                    rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
                except ValueError:
                    pass
        os.unlink(self.path)
        if len(rows) > getattr(self, "skip", 0):
            rows = rows[self.skip:]
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2 + k] == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def peaks():
    try:
        return json.load(open(MEASURED_PEAKS)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# Algorithmic transcendental work of one classic neuron-step (the method's
# count, independent of how a kernel evaluates it): the six rate functions
# and the three gate relaxation factors and V's are ten exponentials; the
# three steady states p_inf = alpha/(alpha+beta) and V's 1/G are four
# divisions.
ALGO_EXP_PER_STEP, ALGO_DIV_PER_STEP = 10, 4


def mufu_ops_per_neuron_step(model):
    """Transcendental work of one exponential-Euler neuron step in the SFU
    formulation, as (exponentials, divisions).  A rate takes one exponential
    per exp/sigmoid/linoid (two for bell) and one division per
    sigmoid/linoid/bell.  An alpha-beta gate adds one division (p_inf); an
    inf-tau or calcium gate's dt/tau takes none for a constant tau, one
    exponential pair and one division for a bell-shaped tau with an offset
    (none without), else the rate's work and one division; a calcium gate's
    p_inf is one division.  Every gate adds one exponential (the relaxation
    factor), and V one division and one exponential.  Classic HH: (10, 7)."""
    work = {"const": (0, 0), "exp": (1, 0), "sigmoid": (1, 1), "linoid": (1, 1), "bell": (2, 1)}
    n_exp = n_div = 0
    for ch in model["channels"]:
        for g in ch["gates"]:
            f1, f2 = g["f1"], g["f2"]
            if g["kind"] == "ab":
                e = work[f1[0]][0] + work[f2[0]][0]
                v = work[f1[0]][1] + work[f2[0]][1] + 1
            else:
                e, v = (0, 1) if g["kind"] == "ca" else work[f1[0]]
                if f2[0] == "bell":
                    e += 2
                    v += 1 if f2[6] != 0.0 else 0
                elif f2[0] != "const":
                    e += work[f2[0]][0]
                    v += work[f2[0]][1] + 1
            n_exp += e + 1
            n_div += v
    return n_exp + 1, n_div + 1


def reduce_over_ranks(ms, spikes, events, world, dev):
    """Replicas only: the job's time is the slowest rank's (MAX), its spikes
    and synaptic events the sum over ranks.  Single process: unchanged."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    tot = torch.tensor([spikes, events], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(t.item()), float(tot[0].item()), float(tot[1].item())


def aggregate_rates(ms_max, spikes_all, events_all, steps, world):
    """Whole-job rates of `world` replicas of the network, each simulating
    `steps` steps of STEPS_PER_SIM time steps (weak scaling): neuron-steps/s,
    synaptic events/s and the mean firing rate in Hz."""
    neuron_steps = float(W["n"]) * STEPS_PER_SIM * steps * world
    value = neuron_steps / (ms_max * 1e-3)
    events_per_s = events_all / (ms_max * 1e-3)
    mean_rate = spikes_all / (W["n"] * world * steps * W["T_ms"] * 1e-3)
    return value, events_per_s, mean_rate


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2601_21407_gb300 import hh

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    # every rank simulates its own replica (independent networks: no data-path collective)
    g = inp.network(n=W["n"], k_in=W["k_in"], exc_frac=W["exc_frac"], seed=W["seed"] + rank,
                    mu=W["mu"], sigma=W["sigma"])
    net = hh.Network(g["V0"], W["dt"], csr=(g["row_ptr"], g["col"], g["w"]), inh=g["inh"], syn=SYN,
                     delay_steps=DELAY, bg=BG, seed=W["seed"] + rank, precision=hh.HH_PREC_FAST,
                     stream=stream.cuda_stream)
    net.set_channels(0, inp.CLASSIC_HH)
    out_deg = np.diff(net.readout(hh.HH_READ_N_OUT))
    out_deg_t = torch.as_tensor(out_deg, device=dev)
    V0_dev = torch.as_tensor(g["V0"], device=dev)
    cap = 8_000_000
    rec, buf = hh.make_record(W["n"], STEPS_PER_SIM, spike_cap=cap, device=dev)

    def step():
        with torch.cuda.stream(stream):
            buf["counts"].zero_()
            buf["n_spikes"].zero_()
        net.reset(V0_dev)
        net.step(STEPS_PER_SIM, rec=rec)

    # launch shape autotuned for this network: each candidate runs one
    # benchmark step (1 s from reset) four times, the median of the last
    # three timed; the state is restored afterwards.  Before the warm-up,
    # outside the timed region.
    net.reset(V0_dev)
    if args.no_autotune:
        tune = {"candidates": [(0, 0, 0.0)], "best": 0}
    else:
        tune = net.autotune(trial_steps=STEPS_PER_SIM)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # SFU and FMA issue rates of this GPU (the roofline denominator of the
    # neuron kernel), measured before the timed region
    sfu_peaks = hh.hh_measure_peaks(stream.cuda_stream)

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    spikes_total = 0
    events_total = 0
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    # activity of the last step (every step simulates the same network from the same state)
    counts = buf["counts"]
    spikes_total = int(counts.sum().item()) * args.steps
    events_total = int((counts.to(torch.int64) * out_deg_t).sum().item()) * args.steps
    status = int(net.readout(hh.HH_READ_STATUS)[0])

    ms_max, spikes_all, events_all = reduce_over_ranks(ms, spikes_total, events_total, world, dev)
    value, events_per_s, mean_rate = aggregate_rates(ms_max, spikes_all, events_all, args.steps, world)

    # kernel timing pass (hh_profile brackets each launch with CUDA events on
    # the network's stream); not part of the timed region above
    net.profile(True)
    step()
    torch.cuda.synchronize()
    kt = net.kernel_times()
    net.profile(False)

    # end-to-end through the public API with host buffers: H2D of the step's
    # initial state from pinned memory, D2H of the spike counts and raster
    V0_host = torch.as_tensor(g["V0"]).pin_memory()
    counts_host = torch.empty(W["n"], dtype=torch.int32).pin_memory()
    spikes_host = torch.empty((cap, 3), dtype=torch.int32).pin_memory()
    nsp_host = torch.empty(1, dtype=torch.int64).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    d2h = 0
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with torch.cuda.stream(stream):
            buf["counts"].zero_()
            buf["n_spikes"].zero_()
        net.reset(V0_host)
        net.step(STEPS_PER_SIM, rec=rec)
        with torch.cuda.stream(stream):
            counts_host.copy_(buf["counts"], non_blocking=True)
            nsp_host.copy_(buf["n_spikes"], non_blocking=True)
        stream.synchronize()
        nsp = min(int(nsp_host.item()), cap)
        with torch.cuda.stream(stream):
            spikes_host[:nsp].copy_(buf["spikes"][:nsp], non_blocking=True)
        stream.synchronize()
        d2h = counts_host.numel() * 4 + 8 + nsp * 12
    e2e_s = time.perf_counter() - t0
    te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = float(W["n"]) * STEPS_PER_SIM * e2e_steps * world / float(te.item())

    # the same network as one cooperative launch per step (comparison)
    persistent_ms = poly_ms = poly_spikes = None
    if rank == 0 and not args.no_extras:
        net2 = hh.Network(g["V0"], W["dt"], csr=(g["row_ptr"], g["col"], g["w"]), inh=g["inh"], syn=SYN,
                          delay_steps=DELAY, bg=BG, seed=W["seed"] + rank, precision=hh.HH_PREC_FAST,
                          stream=stream.cuda_stream, kernels=hh.HH_KERNELS_PERSISTENT)
        net2.set_channels(0, inp.CLASSIC_HH)

        def step2():
            with torch.cuda.stream(stream):
                buf["counts"].zero_()
                buf["n_spikes"].zero_()
            net2.reset(V0_dev)
            net2.step(STEPS_PER_SIM, rec=rec)

        step2()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(2):
            step2()
        f1.record(stream)
        torch.cuda.synchronize()
        persistent_ms = f0.elapsed_time(f1) / 2
        net2.close()
        # the same network on the polynomial rate tables (HH_PREC_POLY)
        net3 = hh.Network(g["V0"], W["dt"], csr=(g["row_ptr"], g["col"], g["w"]), inh=g["inh"], syn=SYN,
                          delay_steps=DELAY, bg=BG, seed=W["seed"] + rank, precision=hh.HH_PREC_POLY,
                          stream=stream.cuda_stream)
        net3.set_channels(0, inp.CLASSIC_HH)

        def step3():
            with torch.cuda.stream(stream):
                buf["counts"].zero_()
                buf["n_spikes"].zero_()
            net3.reset(V0_dev)
            net3.step(STEPS_PER_SIM, rec=rec)

        step3()
        torch.cuda.synchronize()
        f0.record(stream)
        for _ in range(3):
            step3()
        f1.record(stream)
        torch.cuda.synchronize()
        poly_ms = f0.elapsed_time(f1) / 3
        poly_spikes = int(buf["counts"].sum().item())
        net3.close()

    if rank == 0:
        pk, pk_kind = peaks()
        sm_max = float(pk.get("sm_max_mhz", 2070.0))
        n_launch_neuron, neuron_ms = kt["neuron"]
        n_launch_route, route_ms = kt["route"]
        avg_neuron_ms = neuron_ms / max(1, n_launch_neuron)
        steps_per_launch = STEPS_PER_SIM / max(1, n_launch_neuron)
        # the window launch's duration inside the timed schedule: the timed
        # step divided by its window launches (an upper bound on each launch:
        # it includes the routing that co-runs with it and the waits on burst
        # windows), so that launches x duration never exceeds the step
        in_step_ms = (ms_max / args.steps) / max(1, n_launch_neuron)
        assert n_launch_neuron * in_step_ms <= ms_max / args.steps * (1 + 1e-9)
        n_exp, n_div = ALGO_EXP_PER_STEP, ALGO_DIV_PER_STEP
        k_exp, k_div = mufu_ops_per_neuron_step(inp.CLASSIC_HH)
        mufu = n_exp + n_div
        # one cooperative launch per call (routing inside it) or one neuron
        # launch per window with routing launches beside it
        dominant = ("hh_jit_persistent (whole step in one cooperative launch, routing between steps)"
                    if n_launch_route == 0 else "hh_jit_window (k_net_window specialised by NVRTC)")
        ops_per_launch = mufu * W["n"] * steps_per_launch
        achieved_gops = ops_per_launch / (in_step_ms * 1e-3) / 1e9
        # SFU bound of one neuron-step from the measured rates: n_exp
        # ex2.approx and n_div rcp.approx results; the peak is the op count
        # over that time.  The nominal 16 results/clk/SM x sm_max stays in the
        # line for context.
        t_sfu = n_exp / sfu_peaks["ex2_per_s"] + n_div / sfu_peaks["rcp_per_s"]
        peak_gops = mufu / t_sfu / 1e9
        t_sfu_k = k_exp / sfu_peaks["ex2_per_s"] + k_div / sfu_peaks["rcp_per_s"]
        frac_kernel_count = W["n"] * steps_per_launch * t_sfu_k / (in_step_ms * 1e-3)
        nominal_gops = SM_COUNT * MUFU_PER_SM_CLK * sm_max * 1e6 / 1e9
        cpu = cpu_baseline_sample(cores=os.cpu_count()) if not args.no_cpu_baseline else None
        cpu1 = cpu_baseline_sample(cores=1, sim_steps=200) if not args.no_cpu_baseline else None
        line = {
            "metric": "HH neuron-steps/s (conductance-based network, plain FP32 path)",
            "value": value, "unit": "neuron-steps/s", "n_gpus": world, "steps": args.steps,
            "time_steps_per_step": STEPS_PER_SIM,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(),
            "synaptic_events_per_s": events_per_s, "mean_rate_hz": mean_rate,
            "status_bits": status,
            "e2e": {"value": e2e_value, "unit": "neuron-steps/s",
                    "h2d_bytes_per_step": W["n"] * 4, "d2h_bytes_per_step": d2h},
            "gpu_launches": (1 + n_launch_neuron + n_launch_route) * args.steps * world,
            "kernels": {"neuron_window": {"launches_per_step": n_launch_neuron,
                                          "in_step_avg_us": in_step_ms * 1e3,
                                          "profiled_avg_us": avg_neuron_ms * 1e3,
                                          "profiled_schedule": "hh_profile: launch by launch, CUDA events "
                                                               "around each launch (no graph)",
                                          "share_of_step": neuron_ms / max(1e-9, neuron_ms + route_ms)},
                        "route": {"launches_per_step": n_launch_route,
                                  "avg_us": route_ms / max(1, n_launch_route) * 1e3}},
            "roofline": {"bound": "alu", "achieved": achieved_gops, "peak": peak_gops,
                         "unit": "Gop/s (SFU-class: exp + div)",
                         "frac": achieved_gops / peak_gops,
                         "duration_source": "timed step / window launches per step (the launch's share "
                                            "of the timed graph schedule, routing co-running)",
                         # dram__bytes_read.sum + dram__bytes_write.sum of one hh_jit_window
                         # launch (20 steps, cold L2) in an ncu capture of this kernel: the 16 B
                         # of delay line per neuron-step plus the state, nothing re-read
                         "traffic": WINDOW_TRAFFIC_BYTES if (n_launch_route > 0 and WINDOW_TRAFFIC_BYTES) else None,
                         "traffic_unit": "bytes per launch (ncu, cold L2)",
                         "peak_source": f"measured (hh_measure_peaks, all SMs, CUDA events): {n_exp} ex2.approx "
                                        f"+ {n_div} rcp.approx per neuron-step at the measured rates",
                         "nominal_peak": nominal_gops,
                         "nominal_source": f"{SM_COUNT} SMs x {MUFU_PER_SM_CLK} SFU ops/clk x "
                                           f"{sm_max:.0f} MHz ({pk_kind} sm_max)",
                         "ops_per_neuron_step": {"exp": n_exp, "div": n_div,
                                                 "source": "algorithmic count of the classic step"},
                         "frac_at_kernel_op_count": frac_kernel_count,
                         "kernel_ops_per_neuron_step": {"exp": k_exp, "div": k_div},
                         "kernel": dominant},
            "clocks": clk,
            "peaks_measured": {k: v / 1e9 for k, v in sfu_peaks.items()} | {"unit": "G results/s"},
            "launch_shape": {"neuron_block": tune["candidates"][tune["best"]][0],
                             "route_blocks": tune["candidates"][tune["best"]][1],
                             "source": ("the library's default shape (--no-autotune)" if args.no_autotune else
                                        "hh_autotune over one benchmark step (40,000 steps from reset), before "
                                        "the warm-up; (0, 0) is the library's default shape, kept unless another "
                                        "is 3 % faster (median of three timed runs each)"),
                             "sweep_ms_per_step": [list(c) for c in tune["candidates"]]},
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
            line["cpu_baseline_single_core"] = cpu1
        if not args.no_extras:
            line["extra"] = extras(dev, dict(pk, sfu=sfu_peaks))
            if not args.no_batched:
                line["extra"]["batched_64_networks_200ms"] = extra_batched(dev, sfu_peaks)
            line["extra"]["network_persistent_cooperative"] = {
                "ms_per_step": persistent_ms,
                "neuron_steps_per_s": float(W["n"]) * STEPS_PER_SIM / (persistent_ms * 1e-3)}
            line["extra"]["network_poly_rates"] = {
                "ms_per_step": poly_ms, "neuron_steps_per_s": float(W["n"]) * STEPS_PER_SIM / (poly_ms * 1e-3),
                "spikes": poly_spikes, "spikes_plain_path": spikes_total // args.steps,
                "note": "the same workload with HH_PREC_POLY (cubic rate tables fitted at set_channels)"}
        print(json.dumps(line), flush=True)
    net.close()
    if world > 1:
        dist.destroy_process_group()


def sfu_roofline_frac(model, neuron_steps_per_s, peaks):
    """Fraction of the SFU bound of `model` (its exponentials at the measured
    ex2.approx rate plus its divisions at the measured rcp.approx rate)."""
    n_exp, n_div = mufu_ops_per_neuron_step(model)
    return neuron_steps_per_s * (n_exp / peaks["ex2_per_s"] + n_div / peaks["rcp_per_s"])


def bptt_sfu_roofline_frac(model, B, N, T, K, bptt_steps_per_s, peaks):
    """Fraction of the SFU bound of one forward + backward pass of the
    differentiable layer: four passes of T x K neuron-substeps over B x N
    neurons (the forward, the segment recompute, the backward's recompute of
    each outer step's substeps, and the adjoint sweep, whose SFU work per
    substep equals a forward substep's for alpha-beta gates)."""
    n_exp, n_div = mufu_ops_per_neuron_step(model)
    t = 4.0 * T * K * B * N * (n_exp / peaks["ex2_per_s"] + n_div / peaks["rcp_per_s"])
    return bptt_steps_per_s * t


def extra_batched(dev, peaks):
    """The 64 batched heterogeneous networks: sizes LogUniform(1e3, 5e4),
    in-degree U{100..1000}, lognormal weights, half classic and half
    multi-channel networks (7.9e5 neurons, 4.5e8 synapses at seed 0), 1 ms
    delay, background 600 sources x 5 Hz x 1.2 nS, 200 ms (8,000 steps) from
    reset per repetition, launch per 20-step window.  The launch shape is
    autotuned for this network (hh_autotune over the 8,000 steps from reset;
    untimed) and timed against the library's default shape."""
    import torch

    from paper_2601_21407_gb300 import hh
    t_gen = time.perf_counter()
    bn = inp.batched_networks(n_nets=64, seed=0, workers=max(1, min(16, os.cpu_count() or 1)))
    t_gen = time.perf_counter() - t_gen
    N = int(bn["offsets"][-1])
    T = 8_000
    net = hh.Network(bn["V0"], 0.025, csr=(bn["row_ptr"], bn["col"], bn["w"]), inh=bn["inh"], syn=SYN,
                     delay_steps=DELAY, bg={"rate_hz": 5.0, "K": 600, "w": 1.2}, seed=3,
                     precision=hh.HH_PREC_FAST, model_id=bn["model_id"])
    net.set_channels(0, inp.CLASSIC_HH)
    net.set_channels(1, inp.MULTI_CHANNEL)
    V0 = torch.as_tensor(bn["V0"], device=dev)
    out_deg = torch.as_tensor(np.diff(net.readout(hh.HH_READ_N_OUT)), device=dev)
    rec, b = hh.make_record(N, T, spike_cap=0)

    def run():
        b["counts"].zero_()
        net.reset(V0)
        net.step(T, rec=rec)

    def timed_runs(reps=3):
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_default = timed_runs()
    net.reset(V0)
    tune = net.autotune(trial_steps=T)
    ms = timed_runs()
    counts = b["counts"]
    events = float((counts.to(torch.int64) * out_deg).sum().item())
    nc = int((bn["model_id"] == 0).sum())
    frac_c = nc / N
    rate = N * T / (ms * 1e-3)
    # SFU bound of the mix: per-neuron-step time weighted by model share
    t_c = sfu_roofline_frac(inp.CLASSIC_HH, 1.0, peaks)
    t_m = sfu_roofline_frac(inp.MULTI_CHANNEL, 1.0, peaks)
    res = {"neurons": N, "synapses": int(bn["col"].size), "ms_per_200ms_sim": ms,
           "neuron_steps_per_s": rate, "synaptic_events_per_s": events / (ms * 1e-3),
           "mean_rate_hz": float(counts.sum().item()) / N / 0.2,
           "sfu_roofline_frac": rate * (frac_c * t_c + (1 - frac_c) * t_m),
           "graph_generation_s": t_gen, "status": int(net.readout(hh.HH_READ_STATUS)[0]),
           "ms_default_launch_shape": ms_default,
           "launch_shape": {"neuron_block": tune["candidates"][tune["best"]][0],
                            "route_blocks": tune["candidates"][tune["best"]][1]},
           "autotune_sweep_ms_per_run": [list(c) for c in tune["candidates"]]}
    net.close()
    return res


def extra_surrogate(dev, timed):
    """Config 4 with the learned gating surrogate: 1e6 multi-channel neurons,
    500 ms, the MLP (3 layers of width 64, bf16 on the tensor cores, 10-step
    windows) trained on 1e6 windows of the plain integrator (training not
    timed; it learns the correction to one exponential-Euler step over the
    window), against the plain FP32 path on the same GPU, at three settings
    of the per-neuron error estimate (off, and bounds on the correction of
    0.1 mV / 0.004 and 0.01 mV / 0.0005): speed-up, share of neuron-windows
    taken from the MLP, spike-count and spike-time errors against the plain
    path, and counts against the FP64 oracle on 256 sampled neurons."""
    import oracle
    from paper_2601_21407_gb300 import hh
    N, T, dt = 1_000_000, 20_000, 0.025
    y = inp.multi_channel_neurons(N, seed=0)

    def one(err=None):
        net = hh.Network(y["V0"], dt, I_const=y["I"], precision=hh.HH_PREC_FAST)
        net.set_channels(0, inp.MULTI_CHANNEL, gbar=y["gbar"])
        rep = None
        if err is not None:
            rep = net.train_surrogate(v_envelope=-55.0, train_neurons=16384, train_windows=1_000_000,
                                      epochs=30, batch=8192, err_V=err[0], err_p=err[1])
            net.enable_surrogate(True)
        rec, b = hh.make_record(N, T, spike_cap=40 * N)
        net.step(10)
        b["counts"].zero_()
        b["n_spikes"].zero_()
        net.reset()
        ms = timed(lambda: net.step(T, rec=rec))
        acc, dec = net.surrogate_stats() if err is not None else (0, 0)
        out = (b["counts"].cpu().numpy(), hh.spikes_to_numpy(b), ms, acc / max(1, acc + dec), rep)
        net.close()
        return out

    cp, spk_p, plain_ms, _, _ = one()
    idx = np.random.default_rng(1).choice(N, 256, replace=False)
    ref = oracle.simulate(inp.MULTI_CHANNEL, y["I"][idx], y["V0"][idx], T, dt, gbar=y["gbar"][:, idx],
                          trace=False, spk_cap=4)
    res = {"plain_ms": plain_ms,
           "plain_count_within_1_vs_oracle": float((np.abs(cp[idx] - ref["counts"]) <= 1).mean()),
           "settings": []}
    (sp, ip, fp) = spk_p
    for err in ((0.0, 0.0), (0.1, 0.004), (0.01, 0.0005)):
        cs, (ss, is_, fs), ms, acc_frac, rep = one(err)
        d = np.abs(cs.astype(np.int64) - cp)
        # spike times of (a sample of) the neurons whose counts agree
        eq = np.nonzero(d == 0)[0]
        sel = np.random.default_rng(0).choice(eq, min(20_000, eq.size), replace=False) if eq.size else eq
        mp, ms_ = np.isin(ip, sel), np.isin(is_, sel)
        tp = np.lexsort(((sp[mp] + fp[mp]), ip[mp]))
        ts = np.lexsort(((ss[ms_] + fs[ms_]), is_[ms_]))
        dtv = np.abs((sp[mp] + fp[mp])[tp] - (ss[ms_] + fs[ms_])[ts]) * dt
        worst = np.zeros(N)
        np.maximum.at(worst, ip[mp][tp], dtv)
        res["settings"].append({
            "err_V_mV": err[0], "err_p": err[1], "surrogate_ms": ms, "speedup_vs_plain": plain_ms / ms,
            "neuron_steps_per_s": N * T / (ms * 1e-3), "accepted_frac": acc_frac,
            "val_loss": rep["val_loss"],
            "count_equal_vs_plain": float((d == 0).mean()), "count_within_1_vs_plain": float((d <= 1).mean()),
            "max_count_diff_vs_plain": int(d.max()),
            "spike_times_within_0.05ms_of_plain": float((worst[sel] <= 0.05).mean()) if sel.size else None,
            "count_within_1_vs_oracle": float((np.abs(cs[idx] - ref["counts"]) <= 1).mean())})
    res["note"] = ("the MLP corrects one exponential-Euler step over the window; the error estimate bounds "
                   "that correction and trades accepted windows for accuracy: off, the surrogate misses the "
                   "0.05 ms spike-time target; at 0.01 mV it meets the +-1 count / 0.05 ms target on about "
                   "half of the windows; no setting is faster than the plain path (inference is "
                   "latency-bound)")
    return res


def extras(dev, pk):
    """Throughput of the other workloads on the same GPU (not the headline):
    single classic neurons (1,024 x 10,000 steps, dt 0.01 ms), the
    differentiable layer (B=128, 700 inputs, 1,024 neurons, T=250 x 10
    substeps, forward + BPTT), 1e6 multi-channel neurons (20,000 steps,
    dt 0.025 ms), and the tcgen05 GEMM on the layer's two large shapes."""
    import torch

    from paper_2601_21407_gb300 import hh
    out = {}

    def timed(fn, reps=1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    x = inp.single_neurons(1024, seed=0)
    for name, prec in (("compensated", hh.HH_PREC_COMPENSATED), ("fast", hh.HH_PREC_FAST),
                       ("poly", hh.HH_PREC_POLY)):
        net = hh.Network(x["V0"], 0.01, I_const=x["I"], precision=prec)
        net.set_channels(0, inp.CLASSIC_HH)
        rec, b = hh.make_record(1024, 10_000, spike_cap=100_000)
        net.step(10)
        ms = timed(lambda: net.step(10_000, rec=rec), reps=3)
        out[f"single_neurons_1024_{name}"] = {"neuron_steps_per_s": 1024 * 10_000 / (ms * 1e-3),
                                              "ms_per_100ms_sim": ms}
        net.close()

    y = inp.multi_channel_neurons(1_000_000, seed=0)
    for name, prec in (("multichannel_1e6_500ms", hh.HH_PREC_FAST),
                       ("multichannel_1e6_500ms_poly", hh.HH_PREC_POLY)):
        net = hh.Network(y["V0"], 0.025, I_const=y["I"], precision=prec)
        net.set_channels(0, inp.MULTI_CHANNEL, gbar=y["gbar"])
        net.step(10)
        rec, b = hh.make_record(1_000_000, 20_000, spike_cap=0)
        ms = timed(lambda: net.step(20_000, rec=rec))
        out[name] = {"neuron_steps_per_s": 1e6 * 20_000 / (ms * 1e-3), "ms": ms,
                     "mean_rate_hz": float(b["counts"].sum().item()) / 1e6 / 0.5,
                     "sfu_roofline_frac": sfu_roofline_frac(inp.MULTI_CHANNEL, 1e6 * 20_000 / (ms * 1e-3),
                                                            pk["sfu"])}
        if prec == hh.HH_PREC_POLY:
            info = net.readout(hh.HH_READ_POLY)
            out[name]["poly_interval_mV"], out[name]["poly_rel_err"] = float(info[0]), float(info[2])
            out[name]["note"] = ("sfu_roofline_frac: the plain path's SFU work per neuron-step over this "
                                 "path's time (the tables replace most of that work)")
        net.close()
    del y

    out["surrogate_multichannel_1e6_500ms"] = extra_surrogate(dev, timed)

    # frequency-response sweep: 256 frequencies (1-1000 Hz) x 256 amplitudes
    # (up to 20 uA/cm^2), the drive generated in the kernel, 1 s at dt 0.01 ms
    sw = inp.sin_sweep(n_f=256, n_A=256, f_min=1.0, f_max=1000.0, A_max=20.0, I0=0.0)
    Nsw = sw["V0"].size
    net = hh.Network(sw["V0"], 0.01, I_const=sw["I"], precision=hh.HH_PREC_FAST,
                     drive={"amp": sw["amp"], "freq_hz": sw["freq_hz"], "phase": sw["phase"]})
    net.set_channels(0, inp.CLASSIC_HH)
    rec, b = hh.make_record(Nsw, 100_000, spike_cap=0)
    net.step(10)
    b["counts"].zero_()
    net.reset()
    ms = timed(lambda: net.step(100_000, rec=rec))
    rmap = b["counts"].cpu().numpy().reshape(sw["n_A"], sw["n_f"])
    fired = rmap > 0
    thr = [float(np.linspace(20.0 / 256, 20.0, 256)[np.argmax(fired[:, j])]) if fired[:, j].any() else None
           for j in range(sw["n_f"])]
    best = int(np.argmin([t if t is not None else 1e9 for t in thr]))
    out["frequency_response_sweep_65536_1s"] = {
        "neuron_steps_per_s": Nsw * 100_000 / (ms * 1e-3), "ms": ms,
        "points_firing": float(fired.mean()),
        "lowest_threshold_amplitude_uA_cm2": thr[best],
        "at_frequency_hz": float(np.geomspace(1.0, 1000.0, 256)[best]),
        "status": int(net.readout(hh.HH_READ_STATUS)[0])}
    net.close()

    # current-based cortex variant: 77,000 BC2008 cells (80 % RS, 20 % FS),
    # in-degree 1,000 (7.7e7 synapses), current synapses N(0.26, 0.026)
    # uA/cm^2 (inhibitory x 4), compound background 2,000 x 8 Hz x N(0.17,
    # 0.017), dt 0.1 ms, 1.5 ms delay, 1 s simulated
    ct = inp.cortex_network(n=77_000, k_in=1_000, seed=0)
    csyn = {"tau_E": 0.5, "tau_I": 0.5, "E_E": 0.0, "E_I": -80.0, "area_cm2": 2e-4}
    net = hh.Network(ct["V0"], 0.1, csr=(ct["row_ptr"], ct["col"], ct["w"]), inh=ct["inh"], syn=csyn,
                     delay_steps=15, bg={"rate_hz": 8.0, "K": 2000, "w": 0.17, "sd": 0.017}, seed=1,
                     precision=hh.HH_PREC_FAST, model_id=ct["model_id"], syn_mode=hh.HH_SYN_CURRENT)
    net.set_channels(0, inp.BC2008_RS)
    net.set_channels(1, inp.BC2008_FS)
    V0c = torch.as_tensor(ct["V0"], device=dev)
    rec, b = hh.make_record(77_000, 10_000, spike_cap=0)

    def run_ct():
        b["counts"].zero_()
        net.reset(V0c)
        net.step(10_000, rec=rec)

    run_ct()
    ms = timed(run_ct, reps=2)
    cc = b["counts"].cpu().numpy()
    out_deg = np.diff(net.readout(hh.HH_READ_N_OUT))
    out["cortex_current_based_77k_1s"] = {
        "neuron_steps_per_s": 77_000 * 10_000 / (ms * 1e-3), "ms_per_1s_sim": ms,
        "synaptic_events_per_s": float((cc.astype(np.int64) * out_deg).sum()) / (ms * 1e-3),
        "rate_exc_hz": float(cc[:61_600].mean()), "rate_inh_hz": float(cc[61_600:].mean()),
        "status": int(net.readout(hh.HH_READ_STATUS)[0])}
    net.close()
    del ct

    # multi-compartment cells: 65,536 cells of a soma and 3 dendrites x 8
    # compartments (25 of the 32 lanes of a warp), 100 ms at dt 0.01 ms
    cb = inp.cable_cells(65_536, seed=0)
    Ncb = cb["V0"].size
    net = hh.Network(cb["V0"], 0.01, I_const=cb["I"], precision=hh.HH_PREC_FAST, morph=cb["morph"])
    net.set_channels(0, inp.CLASSIC_HH, gbar=cb["gbar"])
    rec, b = hh.make_record(Ncb, 10_000, spike_cap=0)
    net.step(10)
    b["counts"].zero_()
    net.reset()
    ms = timed(lambda: net.step(10_000, rec=rec))
    counts = b["counts"].cpu().numpy().reshape(65_536, 32)
    out["cable_cells_65536x25_100ms"] = {
        "compartment_steps_per_s": 65_536 * cb["n_comp"] * 10_000 / (ms * 1e-3),
        "lane_steps_per_s": Ncb * 10_000 / (ms * 1e-3), "ms": ms,
        "somata_firing": float((counts[:, 0] > 0).mean()),
        "status": int(net.readout(hh.HH_READ_STATUS)[0])}
    net.close()

    d = inp.recurrent_layer(B=128, n_in=700, n_hid=1024, n_out=20, T=250, seed=0)
    lay = hh.Layer(inp.CLASSIC_HH, batch=128, n_in=700, n_hidden=1024, n_out=20, n_steps=250,
                   substeps=10, dt=0.01, precision=hh.HH_PREC_FAST, checkpoint_every=25)
    lay.set_weights(d["W_in"], d["W_rec"], d["W_out"], d["bias"])
    X = torch.as_tensor(d["X"], device=dev)
    lab = torch.as_tensor(d["labels"], device=dev)
    loss = torch.zeros(1, device=dev)
    g = [torch.zeros(s, device=dev) for s in ((700, 1024), (1024, 1024), (20, 1024), (1024,))]
    lay.forward(X, lab, loss)
    lay.backward(*g)
    fwd = timed(lambda: lay.forward(X, lab, loss), reps=3)
    both = timed(lambda: (lay.forward(X, lab, loss), lay.backward(*g)), reps=3)
    out["bptt_layer_b128_t250"] = {"bptt_steps_per_s": 1e3 / both, "forward_ms": fwd,
                                   "backward_ms": both - fwd, "loss": float(loss.item()),
                                   "sfu_roofline_frac": bptt_sfu_roofline_frac(inp.CLASSIC_HH, 128, 1024, 250, 10,
                                                                               1e3 / both, pk["sfu"]),
                                   "status": int(lay.readout(hh.HH_LAYER_STATUS)[0])}
    lay.close()

    peak = float(pk.get("bf16_tflops", 1933.0))
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    for name, (M, N, K, splits) in {"input_projection_32000x1024x704": (32000, 1024, 704, 1),
                                    "weight_grad_1024x704x32000": (1024, 704, 32000, 7)}.items():
        A = torch.randn(M, K, device=dev).to(torch.bfloat16)
        Bt = torch.randn(N, K, device=dev).to(torch.bfloat16)
        Cc = torch.empty((splits, M, N), device=dev)
        hh.hh_gemm_bf16(A, Bt, Cc, M, N, K, splits=splits, status=st)
        ms = timed(lambda: hh.hh_gemm_bf16(A, Bt, Cc, M, N, K, splits=splits, status=st), reps=10)
        tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
        out[f"gemm_{name}"] = {"tflops": tf, "frac_of_measured_bf16": tf / peak, "us": ms * 1e3}
    return out


def cpu_baseline_sample(cores, sim_steps=None):
    """The FP64 oracle on the host cores: the full 38,000-neuron network for a
    bounded number of time steps (default 2,000 = 50 ms), timed as the
    difference of a run with and without the steps (graph transposition and
    allocation excluded)."""
    import oracle
    sim_steps = sim_steps or int(os.environ.get("HH_CPU_SAMPLE_STEPS", "2000"))
    g = inp.network(n=W["n"], k_in=W["k_in"], exc_frac=W["exc_frac"], seed=W["seed"],
                    mu=W["mu"], sigma=W["sigma"])
    t0 = time.perf_counter()
    oracle.simulate_network(inp.CLASSIC_HH, g, 1, W["dt"], DELAY, SYN, bg=BG, seed=W["seed"],
                            spk_cap=4, n_threads=cores)
    base = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = oracle.simulate_network(inp.CLASSIC_HH, g, sim_steps + 1, W["dt"], DELAY, SYN, bg=BG,
                                seed=W["seed"], spk_cap=4, n_threads=cores)
    full = time.perf_counter() - t0
    dt_s = max(1e-9, full - base)
    return {"value": W["n"] * sim_steps / dt_s, "unit": "neuron-steps/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{sim_steps} time steps ({sim_steps * W['dt']:.0f} ms) of the full "
                      f"38,000-neuron network, FP64, OpenMP over neurons ({cores} thread{'s' if cores != 1 else ''}); "
                      f"{int(r['counts'].sum())} spikes"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count()
    sample_steps = int(os.environ.get("HH_REF_SAMPLE_STEPS", "400"))
    import oracle
    g = inp.network(n=W["n"], k_in=W["k_in"], exc_frac=W["exc_frac"], seed=W["seed"],
                    mu=W["mu"], sigma=W["sigma"])

    def run(n):
        t0 = time.perf_counter()
        oracle.simulate_network(inp.CLASSIC_HH, g, n, W["dt"], DELAY, SYN, bg=BG,
                                seed=W["seed"], spk_cap=4, n_threads=cores)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        run(sample_steps + 1)
    # the oracle's set-up (graph transposition, allocation) as the time of a
    # one-step run, subtracted from each step as in the CPU-baseline leg
    base = min(run(1) for _ in range(2))
    times = [max(1e-9, run(sample_steps + 1) - base) for _ in range(args.steps)]
    tot = sum(times)
    value = W["n"] * sample_steps * args.steps / tot
    line = {"impl": "reference", "metric": "HH neuron-steps/s (conductance-based network, plain FP32 path)",
            "value": value, "unit": "neuron-steps/s", "n_gpus": world, "steps": args.steps,
            "time_steps_per_step": sample_steps,
            "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": "neuron-steps/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"each step: {sample_steps} time steps of the full 38,000-neuron "
                                       f"network, FP64, OpenMP over neurons; the oracle's set-up (a one-step "
                                       f"run, {base:.2f} s) subtracted"},
            "e2e": {"value": value, "unit": "neuron-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def ncu_case(name):
    """Small fixed cases for ncu captures.
    network: the benchmark network, 120 time steps (six 20-step windows,
             one neuron and one routing launch each), then one open-loop
             routing launch of a 40-step raster with 1% of the neurons
             spiking per step;
    network-persistent: the same with the 120 steps in one cooperative
             launch;
    multichannel: 1e6 multi-channel neurons, two launches of 200 steps;
    gemm:    the layer's input projection (32000 x 1024 x 704, bf16) twice;
    layer:   the differentiable layer at full width (B=128, 700 inputs, 1,024
             neurons) for T=25 outer steps, forward and backward."""
    import torch

    from paper_2601_21407_gb300 import hh
    torch.cuda.set_device(0)
    if name == "multichannel":
        y = inp.multi_channel_neurons(1_000_000, seed=0)
        net = hh.Network(y["V0"], 0.025, I_const=y["I"], precision=hh.HH_PREC_FAST)
        net.set_channels(0, inp.MULTI_CHANNEL, gbar=y["gbar"])
        rec, b = hh.make_record(1_000_000, 200, spike_cap=0)
        for _ in range(2):
            net.step(200, rec=rec)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": "multichannel", "status": int(net.readout(hh.HH_READ_STATUS)[0])}))
        net.close()
        return
    if name == "gemm":
        M, N, K = 32000, 1024, 704
        A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
        Bt = torch.randn(N, K, device="cuda").to(torch.bfloat16)
        Cc = torch.empty((1, M, N), device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        for _ in range(2):
            hh.hh_gemm_bf16(A, Bt, Cc, M, N, K, status=st)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": "gemm", "status": int(st.item())}))
        return
    if name == "layer":
        d = inp.recurrent_layer(B=128, n_in=700, n_hid=1024, n_out=20, T=25, seed=0)
        lay = hh.Layer(inp.CLASSIC_HH, batch=128, n_in=700, n_hidden=1024, n_out=20, n_steps=25,
                       substeps=10, dt=0.01, precision=hh.HH_PREC_FAST, checkpoint_every=25)
        lay.set_weights(d["W_in"], d["W_rec"], d["W_out"], d["bias"])
        X = torch.as_tensor(d["X"], device="cuda")
        lab = torch.as_tensor(d["labels"], device="cuda")
        loss = torch.zeros(1, device="cuda")
        g = [torch.zeros(s, device="cuda") for s in ((700, 1024), (1024, 1024), (20, 1024), (1024,))]
        lay.forward(X, lab, loss)
        lay.backward(*g)
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": "layer", "loss": float(loss.item()),
                          "status": int(lay.readout(hh.HH_LAYER_STATUS)[0])}))
        lay.close()
        return
    g = inp.network(n=W["n"], k_in=W["k_in"], exc_frac=W["exc_frac"], seed=W["seed"],
                    mu=W["mu"], sigma=W["sigma"])
    kernels = hh.HH_KERNELS_PERSISTENT if name == "network-persistent" else hh.HH_KERNELS_SPECIALISED
    net = hh.Network(g["V0"], W["dt"], csr=(g["row_ptr"], g["col"], g["w"]), inh=g["inh"], syn=SYN,
                     delay_steps=DELAY, bg=BG, seed=W["seed"], precision=hh.HH_PREC_FAST, kernels=kernels)
    net.set_channels(0, inp.CLASSIC_HH)
    rec, b = hh.make_record(W["n"], 3 * DELAY, spike_cap=100_000)
    net.step(3 * DELAY, rec=rec)
    st, ix = inp.spike_raster(W["n"], DELAY, W["n"] // 100, 1)
    sE = torch.zeros((2 * DELAY, W["n"]), dtype=torch.int64, device="cuda")
    sI = torch.zeros_like(sE)
    net.route_spikes(torch.as_tensor(st, device="cuda"), torch.as_tensor(ix, device="cuda"),
                     2 * DELAY, sE, sI)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": "network38k", "spikes": int(b["n_spikes"].item()),
                      "raster_events": int(len(st)) * W["k_in"]}))
    net.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default launch shape (no hh_autotune before the warm-up; the launch "
                         "indices of the timed steps are then those of the profiles' ncu commands)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 64 batched heterogeneous networks (graph generation on the host cores)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other workloads (single neurons, BPTT layer, 1e6 neurons, GEMM)")
    ap.add_argument("--ncu-case", nargs="?", const="network", default=None,
                    choices=["network", "network-persistent", "multichannel", "gemm", "layer"],
                    help="run a small fixed case used for ncu captures and exit")
    args = ap.parse_args()
    if args.ncu_case:
        ncu_case(args.ncu_case)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
