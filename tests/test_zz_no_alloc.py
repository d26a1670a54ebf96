"""hh_step_neurons_noalloc: stepping independent neurons in buffers the caller
already owns, for callers that cannot call cudaMalloc themselves (code that
lives inside another framework's memory pool or arena, or a process that must
not grow its device footprint once it is running).  The entry point keeps its
only scratch space -- the neuron -> V-trace-slot map -- in a static device
array of the library, so it allocates nothing.

Checked through the C ABI against the allocating path (hh_create_network +
hh_step_n) on two calls in a row, within the tolerances the other GPU tests
use (V within 1e-2 mV, identical spike counts and rasters), and the device's
free memory is the same before and after the second call.  The allocating
path runs the same precompiled table kernels (HH_KERNELS_TABLE) as the
entry point: loading run-time compiled kernels allocates device memory, and
two compilations of the step may contract different multiply-adds, whose
ulp-level difference drifts the phase of a regularly firing neuron over
thousands of steps.  This file is
collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

from paper_2601_21407_gb300 import hh, inputs as inp

pytestmark = pytest.mark.gpu

V_TOL_MV = 1e-2


def _torch():
    import torch
    return torch


def _record(N, T, trace_idx):
    return hh.make_record(N, T, trace=len(trace_idx), trace_idx=trace_idx, spike_cap=200_000)


@pytest.mark.parametrize("prec,with_status", [(hh.HH_PREC_COMPENSATED, True),
                                              (hh.HH_PREC_FAST, False)])
def test_noalloc_matches_allocating_path(prec, with_status):
    torch = _torch()
    torch.cuda.set_device(0)
    N = 777
    x = inp.single_neurons(N, seed=11)
    dt = 0.01
    steps = (1500, 2300)
    trace_idx = np.random.default_rng(3).permutation(N)[:300].astype(np.int32)

    # allocating path: the library owns the state
    net = hh.Network(x["V0"], dt, I_const=x["I"], precision=prec, kernels=hh.HH_KERNELS_TABLE)
    net.set_channels(0, inp.CLASSIC_HH)
    ref = []
    for T in steps:
        rec, b = _record(N, T, trace_idx)
        net.step(T, rec=rec)
        torch.cuda.synchronize()
        ref.append((b["V_trace"].cpu().numpy(), b["counts"].cpu().numpy(), hh.spikes_to_numpy(b)))
    net.close()

    # allocation-free path: the caller owns every buffer (allocated here by
    # the test, never by the entry point)
    dev = "cuda"
    V = torch.as_tensor(x["V0"], device=dev).clone()
    gates = torch.zeros((hh.HH_MAX_GATES, N), dtype=torch.float32, device=dev)
    Ca = torch.zeros(N, dtype=torch.float32, device=dev)
    V_lo = torch.zeros_like(V)
    gates_lo = torch.zeros_like(gates)
    I_const = torch.as_tensor(x["I"], device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    s = hh.hh_neurons_noalloc()
    s.n_neurons = N
    s.dt_ms = dt
    s.v_threshold = 0.0
    s.v_update = hh.HH_V_EXP_EULER
    s.precision = prec
    s.V, s.gates, s.Ca = V.data_ptr(), gates.data_ptr(), Ca.data_ptr()
    if prec == hh.HH_PREC_COMPENSATED:
        s.V_lo, s.gates_lo = V_lo.data_ptr(), gates_lo.data_ptr()
    s.I_const = I_const.data_ptr()
    s.status = status.data_ptr() if with_status else None
    m = hh.model_desc(inp.CLASSIC_HH)
    t0 = 0
    for call, T in enumerate(steps):
        s.init_state = 1 if call == 0 else 0
        rec, b = _record(N, T, trace_idx)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        hh.hh_step_neurons_noalloc(m, s, t0, T, None, rec)
        torch.cuda.synchronize()
        if call > 0:
            # the first call may load the library's kernels (lazy module
            # loading reserves device memory once); later calls take none
            assert torch.cuda.mem_get_info()[0] == free_before
        t0 += T
        Vtr = b["V_trace"].cpu().numpy()
        Vref, cref, sref = ref[call]
        assert np.abs(Vtr - Vref).max() <= V_TOL_MV
        assert np.array_equal(b["counts"].cpu().numpy(), cref)
        got = hh.spikes_to_numpy(b)
        assert np.array_equal(got[0], sref[0]) and np.array_equal(got[1], sref[1])
        assert np.abs(got[2] - sref[2]).max() <= 1e-3
    assert sum(int(c.sum()) for _, c, _ in ref) > 100
    if with_status:
        assert int(status.item()) == 0


def test_noalloc_rejects_oversize():
    s = hh.hh_neurons_noalloc()
    s.n_neurons = hh.HH_NOALLOC_MAX_NEURONS + 1
    s.dt_ms = 0.01
    with pytest.raises(hh.HHError) as e:
        hh.hh_step_neurons_noalloc(hh.model_desc(inp.CLASSIC_HH), s, 0, 10)
    assert e.value.status == hh.HH_EINVAL
    assert "static scratch" in str(e.value)
