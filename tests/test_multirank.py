"""The N > 1 path of bench.py, on CPU with the gloo backend (world size 2).

Every rank simulates its own replica of the network (independent networks,
no data-path collective): the job's time is the slowest rank's, its spikes
and synaptic events add up, and the whole-job rate counts the neuron-steps
of all replicas.  The reference (oracle) arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [40.0, 55.0][rank]
        spikes = [1000.0, 3000.0][rank]
        events = [2.0e6, 5.0e6][rank]
        ms_max, spikes_all, events_all = bench.reduce_over_ranks(ms, spikes, events, world, "cpu")
        value, events_per_s, rate = bench.aggregate_rates(ms_max, spikes_all, events_all, steps=2,
                                                          world=world)
        q.put((rank, ms_max, spikes_all, events_all, value, events_per_s, rate))
    finally:
        dist.destroy_process_group()


def test_replicas_reduce_max_time_and_sum_counts():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    sys.path.insert(0, ROOT)
    import bench
    n_steps = bench.W["n"] * bench.STEPS_PER_SIM * 2 * world
    for rank, ms_max, spikes_all, events_all, value, events_per_s, rate in res:
        assert ms_max == 55.0
        assert spikes_all == 4000.0 and events_all == 7.0e6
        assert value == pytest.approx(n_steps / 55e-3)
        assert events_per_s == pytest.approx(7.0e6 / 55e-3)
        assert rate == pytest.approx(4000.0 / (bench.W["n"] * world * 2 * bench.W["T_ms"] * 1e-3))


def test_reference_arm_only_on_rank_zero(monkeypatch, capsys):
    """A rank other than 0 returns from the oracle arm without work or output."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup = 1, 3

    bench.run_reference(Args())
    assert capsys.readouterr().out == ""
