"""Host-side pieces that need no GPU: the benchmark's work counting and
oracle arm, and the autograd wrapper's own logic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2601_21407_gb300 import inputs as inp  # noqa: E402


def test_sfu_work_per_neuron_step():
    """Classic HH: 6 rate exponentials + 3 gate and 1 membrane relaxation
    factors = 10; 2 linoid + 1 sigmoid rate divisions + 3 p_inf + 1 V_inf = 7.
    Multi-channel: the bell-shaped time constants of KA (offsets 0.37 and 19
    ms) take one division each and that of Ih (no offset) none; KCa's
    constant time constant none."""
    assert bench.mufu_ops_per_neuron_step(inp.CLASSIC_HH) == (10, 7)
    assert bench.mufu_ops_per_neuron_step(inp.MULTI_CHANNEL) == (26, 16)


def test_reference_arm_line(monkeypatch, capsys):
    """The oracle arm prints one JSON line with the contract's keys, on the
    benchmark's workload and metric, with the oracle's set-up subtracted."""
    import json
    monkeypatch.setenv("HH_REF_SAMPLE_STEPS", "4")
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")

    class Args:
        steps, warmup = 1, 3

    bench.run_reference(Args())
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    r = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in r, k
    assert r["impl"] == "reference" and r["dtype"] == "f64" and r["value"] > 0
    assert r["config"] == bench.workload_config()
    assert r["cpu_baseline"]["kind"] == "oracle" and r["cpu_baseline"]["value"] == r["value"]
    assert r["e2e"]["value"] == r["value"] and r["e2e"]["h2d_bytes_per_step"] == 0
    assert "subtracted" in r["cpu_baseline"]["sample"]


def test_layer_function_host_logic():
    """The autograd wrapper's own logic, on a stand-in for the library layer
    (CPU tensors): the weights go to set_weights before the forward, the
    incoming gradient of the loss becomes the built-in loss's weight and the
    incoming gradient of the logits the dL/dlogits cotangent, the spike
    inputs and labels get no gradient, and a second forward makes the first
    graph's backward raise."""
    import pytest
    import torch

    from paper_2601_21407_gb300 import hh

    class FakeLayer:
        shape = (5, 2, 3, 4, 2)  # T, B, n_in, N, n_out
        _forward_id = 0

        def set_weights(self, *w):
            self.w = [x.clone() for x in w]

        def forward(self, X, labels, loss, logits):
            loss.fill_(float(sum(x.sum() for x in self.w)))
            logits.fill_(1.0)
            self._forward_id += 1

        def backward_from(self, *, ce_weight, dL_dlogits, dW_in, dW_rec, dW_out, dbias):
            extra = 0.0 if dL_dlogits is None else float(dL_dlogits.sum())
            for k, x in enumerate((dW_in, dW_rec, dW_out, dbias)):
                x.fill_((k + 1.0) * ce_weight + extra)

    lay = FakeLayer()
    W = [torch.randn(s, requires_grad=True) for s in ((3, 4), (4, 4), (2, 4), (4,))]
    X = torch.zeros((5, 2, 3))
    y = torch.zeros(2, dtype=torch.int32)
    loss, logits = hh.layer_function().apply(lay, X, y, *W)
    assert torch.equal(lay.w[1], W[1].detach())
    assert loss.requires_grad and logits.requires_grad
    (3.0 * loss).backward()
    for k, w in enumerate(W):
        assert torch.equal(w.grad, torch.full_like(w, 3.0 * (k + 1)))
    for w in W:
        w.grad = None
    loss, logits = hh.layer_function().apply(lay, X, y, *W)
    (2.0 * logits.sum()).backward()
    for w in W:
        assert torch.equal(w.grad, torch.full_like(w, 2.0 * 4))
    a, _ = hh.layer_function().apply(lay, X, y, *W)
    b, _ = hh.layer_function().apply(lay, X, y, *W)
    with pytest.raises(RuntimeError):
        a.backward()
    b.backward()


def test_layer_spikes_function_host_logic():
    """The spike-output wrapper on a stand-in layer: the forward runs without
    labels and returns the layer's S and V_T; the backward hands the incoming
    gradients over as dL/dS and dL/dV and returns dX and the weight
    gradients, with dX requested only when X needs it."""
    import torch

    from paper_2601_21407_gb300 import hh

    class FakeLayer:
        shape = (5, 2, 3, 4, 2)
        _forward_id = 0

        def set_weights(self, *w):
            self.w = [x.clone() for x in w]

        def forward(self, X, labels=None, loss=None, logits=None):
            assert labels is None and loss is None
            self.X = X.clone()
            self._forward_id += 1

        def outputs(self, S, V):
            S.fill_(1.0)
            V.fill_(-60.0)

        def backward_from(self, *, dL_dS, dL_dV, dW_in, dW_rec, dbias, dX):
            self.got = (dL_dS.clone(), dL_dV.clone(), dX is not None)
            for k, x in enumerate((dW_in, dW_rec, dbias)):
                x.fill_(float(dL_dS.sum()) + k)
            if dX is not None:
                dX.fill_(7.0)

    lay = FakeLayer()
    W_in, W_rec, bias = [torch.randn(s, requires_grad=True) for s in ((3, 4), (4, 4), (4,))]
    Z = torch.zeros((5, 2, 3), requires_grad=True)
    S, V = hh.layer_spikes_function().apply(lay, 2.0 * Z, W_in, W_rec, bias)
    assert S.shape == (5, 2, 4) and V.shape == (2, 4) and float(V[0, 0]) == -60.0
    (S.sum() + 0.5 * V.sum()).backward()
    dS, dV, want_dx = lay.got
    assert want_dx and float(dS.sum()) == 40.0 and float(dV.sum()) == 4.0
    assert torch.equal(Z.grad, torch.full_like(Z, 14.0))
    assert torch.equal(W_rec.grad, torch.full_like(W_rec, 41.0))


def test_bptt_sfu_bound():
    """One forward + backward of the 128 x 1,024-neuron layer over 250 x 10
    substeps is four passes of 3.28e8 classic neuron-substeps (10 ex2 + 7
    rcp each): 3.15 ms at 1e13 ex2/s and 5e12 rcp/s, so 69 passes per
    second sit at 21.7 % of that bound."""
    pk = {"ex2_per_s": 1e13, "rcp_per_s": 5e12}
    t = bench.bptt_sfu_roofline_frac(inp.CLASSIC_HH, 128, 1024, 250, 10, 1.0, pk)
    assert abs(t - 4 * 250 * 10 * 128 * 1024 * (10 / 1e13 + 7 / 5e12)) < 1e-12
    assert abs(bench.bptt_sfu_roofline_frac(inp.CLASSIC_HH, 128, 1024, 250, 10, 69.0, pk) - 0.2171) < 1e-3


def test_cpu_baseline_sample_single_core():
    """The oracle timed on one host thread: the baseline dict the bench line
    carries (value, unit, cores, kind, sample)."""
    r = bench.cpu_baseline_sample(cores=1, sim_steps=5)
    assert r["cores"] == 1 and r["kind"] == "oracle" and r["unit"] == "neuron-steps/s"
    assert r["value"] > 0 and "(1 thread)" in r["sample"]
