"""GPU parity of the differentiable recurrent HH layer (hh_layer_* and
hh_backward via the C ABI) against the FP64 autograd oracle: spike rasters,
loss, logits and the gradients of W_in, W_rec, W_out and bias, in the
surrogate (Heaviside) and smooth-spike programs; the full-size layer
(B=128, 700 inputs, 1,024 neurons, T=250 x 10 substeps) on sampled batch
elements."""
import numpy as np
import pytest

from oracle import bptt
from paper_2601_21407_gb300 import hh, inputs as inp

pytestmark = pytest.mark.gpu

HH = inp.CLASSIC_HH


def _torch():
    import torch
    return torch


def run_layer(d, *, T, B, n_in, N, n_out, K=10, dt=0.01, precision=hh.HH_PREC_ACCURATE, smooth=False,
              ckpt=7, backward=True):
    torch = _torch()
    lay = hh.Layer(HH, batch=B, n_in=n_in, n_hidden=N, n_out=n_out, n_steps=T, substeps=K, dt=dt,
                   precision=precision, smooth=smooth, checkpoint_every=ckpt)
    lay.set_weights(d["W_in"], d["W_rec"], d["W_out"], d["bias"])
    X = torch.as_tensor(d["X"], device="cuda")
    y = torch.as_tensor(d["labels"], device="cuda")
    loss = torch.zeros(1, device="cuda")
    logits = torch.zeros((B, n_out), device="cuda")
    lay.forward(X, y, loss, logits)
    out = {}
    if backward:
        g = {k: torch.zeros(s, device="cuda") for k, s in
             (("W_in", (n_in, N)), ("W_rec", (N, N)), ("W_out", (n_out, N)), ("bias", (N,)))}
        lay.backward(g["W_in"], g["W_rec"], g["W_out"], g["bias"])
        torch.cuda.synchronize()
        out.update({"d" + k: v.cpu().numpy() for k, v in g.items()})
    torch.cuda.synchronize()
    out["loss"] = float(loss.item())
    out["logits"] = logits.cpu().numpy()
    out["spikes"] = lay.readout(hh.HH_LAYER_SPIKES).reshape(T, B, N)
    out["status"] = int(lay.readout(hh.HH_LAYER_STATUS)[0])
    lay.close()
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def small_case(seed, T=30, B=4, n_in=40, N=64, n_out=5, w_rec=2.0):
    d = inp.recurrent_layer(B=B, n_in=n_in, n_hid=N, n_out=n_out, T=T, seed=seed, rate_max_hz=400.0,
                            w_in_scale=60.0, w_rec_scale=w_rec)
    return d


@pytest.mark.parametrize("precision", [hh.HH_PREC_ACCURATE, hh.HH_PREC_FAST])
def test_layer_surrogate_matches_oracle(precision):
    """Heaviside spikes with the fast-sigmoid surrogate: identical spike
    raster, loss and logits to 1e-5, gradients to 1e-3 (relative, norm-wise)."""
    T, B, n_in, N, n_out = 30, 4, 40, 64, 5
    d = small_case(1, T, B, n_in, N, n_out)
    g = run_layer(d, T=T, B=B, n_in=n_in, N=N, n_out=n_out, precision=precision)
    ref = bptt.layer_grads(HH, d["X"], d["W_in"], d["W_rec"], d["W_out"], d["bias"], d["labels"],
                           K=10, dt=0.01)
    assert g["status"] == 0
    assert ref["spikes"].sum() > 20
    assert np.array_equal(g["spikes"], ref["spikes"])
    assert abs(g["loss"] - ref["loss"]) <= 1e-5 * max(1.0, abs(ref["loss"]))
    assert np.abs(g["logits"] - ref["logits"]).max() <= 1e-5
    for k in ("dW_in", "dW_rec", "dW_out", "dbias"):
        assert rel(g[k], ref[k]) <= 1e-3, (k, rel(g[k], ref[k]))


def test_layer_smooth_matches_oracle():
    """Smooth spikes (a differentiable program pinned by central differences
    in the oracle) without recurrence: loss and every gradient agree with the
    FP64 reverse mode to 1e-3."""
    T, B, n_in, N, n_out = 20, 3, 24, 32, 4
    d = small_case(2, T, B, n_in, N, n_out)
    d["W_rec"] = np.zeros_like(d["W_rec"])
    g = run_layer(d, T=T, B=B, n_in=n_in, N=N, n_out=n_out, smooth=True, ckpt=6)
    ref = bptt.layer_grads(HH, d["X"], d["W_in"], d["W_rec"], d["W_out"], d["bias"], d["labels"],
                           K=10, dt=0.01, smooth=True)
    assert abs(g["loss"] - ref["loss"]) <= 1e-5 * max(1.0, abs(ref["loss"]))
    for k in ("dW_in", "dW_out", "dbias"):
        assert rel(g[k], ref[k]) <= 1e-3, (k, rel(g[k], ref[k]))


def test_layer_checkpoint_interval_invariance():
    """The gradients do not depend on the checkpoint interval (recompute
    reproduces the forward states bit for bit)."""
    T, B, n_in, N, n_out = 26, 2, 16, 32, 3
    d = small_case(3, T, B, n_in, N, n_out)
    a = run_layer(d, T=T, B=B, n_in=n_in, N=N, n_out=n_out, ckpt=1)
    b = run_layer(d, T=T, B=B, n_in=n_in, N=N, n_out=n_out, ckpt=25)
    for k in ("dW_in", "dW_rec", "dW_out", "dbias"):
        assert np.array_equal(a[k], b[k]), k


def test_layer_full_size_sampled():
    """Config 3 at full size on the GPU (B=128, 700 inputs, 1,024 neurons,
    T=250, 10 substeps, checkpoints every 25): the oracle recomputes two
    batch elements alone (samples are independent) and their spike rasters
    and logits agree; gradients are finite and the loss is the mean of the
    per-sample losses."""
    torch = _torch()
    T, B, n_in, N, n_out = 250, 128, 700, 1024, 20
    d = inp.recurrent_layer(B=B, n_in=n_in, n_hid=N, n_out=n_out, T=T, seed=0)
    g = run_layer(d, T=T, B=B, n_in=n_in, N=N, n_out=n_out, precision=hh.HH_PREC_FAST, ckpt=25)
    assert g["status"] == 0
    for k in ("dW_in", "dW_rec", "dW_out", "dbias"):
        assert np.isfinite(g[k]).all() and np.abs(g[k]).max() > 0
    idx = [0, 77]
    with torch.no_grad():
        loss, aux = bptt.layer_forward(HH, torch.tensor(d["X"][:, idx], dtype=torch.float64),
                                       torch.tensor(d["W_in"], dtype=torch.float64),
                                       torch.tensor(d["W_rec"], dtype=torch.float64),
                                       torch.tensor(d["W_out"], dtype=torch.float64),
                                       torch.tensor(d["bias"], dtype=torch.float64),
                                       torch.tensor(d["labels"][idx], dtype=torch.long),
                                       K=10, dt=0.01, return_all=True)
    sp = aux["spikes"].numpy()
    assert sp.sum() > 100
    agree = (g["spikes"][:, idx] == sp).mean()
    assert agree >= 0.9999, agree
    assert np.abs(g["logits"][idx] - aux["logits"].numpy()).max() <= 2e-3


def test_layer_autograd_function():
    """loss.backward() through the torch.autograd.Function gives exactly the
    gradients of hh_backward (the same kernels), scaled by the incoming
    gradient; the spike inputs get none; after a second forward the first
    graph's backward raises."""
    torch = _torch()
    T, B, n_in, N, n_out = 20, 3, 16, 32, 4
    d = small_case(1, T, B, n_in, N, n_out)
    lay = hh.Layer(HH, batch=B, n_in=n_in, n_hidden=N, n_out=n_out, n_steps=T, substeps=10, dt=0.01,
                   precision=hh.HH_PREC_FAST, checkpoint_every=7)
    W = [torch.tensor(d[k], dtype=torch.float32, device="cuda", requires_grad=True)
         for k in ("W_in", "W_rec", "W_out", "bias")]
    X = torch.as_tensor(d["X"], device="cuda")
    y = torch.as_tensor(d["labels"], device="cuda")
    loss, logits = lay.loss(X, y, *W)
    assert loss.requires_grad and not logits.requires_grad
    (2.5 * loss).backward()
    lay.set_weights(*[w.detach() for w in W])
    l2 = torch.zeros(1, device="cuda")
    lay.forward(X, y, l2)
    g = [torch.zeros_like(w) for w in W]
    lay.backward(*g)
    torch.cuda.synchronize()
    assert float(loss.item()) == float(l2.item())
    assert all(float(x.abs().max()) > 0 for x in g)
    for w, gd in zip(W, g):
        assert torch.equal(w.grad, 2.5 * gd)
    loss_a, _ = lay.loss(X, y, *W)
    loss_b, _ = lay.loss(X, y, *W)
    with pytest.raises(RuntimeError):
        loss_a.backward()
    loss_b.backward()
    lay.close()
