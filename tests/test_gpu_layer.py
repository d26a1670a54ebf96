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
    gradients of hh_backward_from with the incoming gradient of the loss as
    the weight of the built-in cross-entropy (the same kernels); the logits
    are differentiable too; the spike inputs get no gradient; after a second
    forward the first graph's backward raises."""
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
    assert loss.requires_grad and logits.requires_grad
    (2.5 * loss).backward()
    lay.set_weights(*[w.detach() for w in W])
    l2 = torch.zeros(1, device="cuda")
    lay.forward(X, y, l2)
    g = [torch.zeros_like(w) for w in W]
    lay.backward_from(ce_weight=2.5, dW_in=g[0], dW_rec=g[1], dW_out=g[2], dbias=g[3])
    torch.cuda.synchronize()
    assert float(loss.item()) == float(l2.item())
    assert all(float(x.abs().max()) > 0 for x in g)
    for w, gd in zip(W, g):
        assert torch.equal(w.grad, gd)
    # a loss of the logits alone flows through dL/dlogits
    for w in W:
        w.grad = None
    loss, logits = lay.loss(X, y, *W)
    R = torch.randn_like(logits)
    (logits * R).sum().backward()
    lay.set_weights(*[w.detach() for w in W])
    lay.forward(X, y, l2)
    g = [torch.zeros_like(w) for w in W]
    lay.backward_from(dL_dlogits=R, dW_in=g[0], dW_rec=g[1], dW_out=g[2], dbias=g[3])
    torch.cuda.synchronize()
    for w, gd in zip(W, g):
        assert torch.equal(w.grad, gd)
    loss_a, _ = lay.loss(X, y, *W)
    loss_b, _ = lay.loss(X, y, *W)
    with pytest.raises(RuntimeError):
        loss_a.backward()
    loss_b.backward()
    lay.close()


def _elementwise(got, ref, tol):
    """max |got - ref| / max |ref| (the bound the tests assert per entry)."""
    scale = max(float(np.abs(ref).max()), 1e-30)
    return float(np.abs(got - ref).max()) / scale


@pytest.mark.parametrize("precision,tol", [(hh.HH_PREC_ACCURATE, 2e-3), (hh.HH_PREC_FAST, 2e-3)])
def test_layer_backward_from_matches_oracle(precision, tol):
    """hh_backward_from with caller cotangents dL/dS [T][B][N] and dL/dV [B][N]
    (no built-in loss): dX, dI, dW_in, dW_rec and dbias agree with the FP64
    oracle's reverse mode element by element, |got - ref| <= tol * max|ref|
    for every entry (measured 0.6-1.0e-3 in both precisions: the FP32
    state's rounding, not the rate arithmetic), on an identical spike
    raster.  The inputs keep every
    substep at least 1e-3 mV from theta in the oracle's trajectory: the
    surrogate gradient jumps where a crossing moves to the next substep, and a
    trajectory passing within FP32 rounding of theta can do that."""
    torch = _torch()
    T, B, n_in, N, n_out = 30, 4, 40, 64, 5
    d = small_case(5, T, B, n_in, N, n_out)
    # conditioning from the oracle alone: no substep within 1e-3 mV of theta,
    # so FP32 and FP64 put every crossing in the same substep
    assert bptt.threshold_margin(HH, d["X"], d["W_in"], d["W_rec"], d["bias"]).min() >= 1e-3
    rng = np.random.default_rng(9)
    dS = rng.normal(0, 1.0, (T, B, N)).astype(np.float32)
    dV = rng.normal(0, 0.05, (B, N)).astype(np.float32)
    lay = hh.Layer(HH, batch=B, n_in=n_in, n_hidden=N, n_out=n_out, n_steps=T, substeps=10, dt=0.01,
                   precision=precision, checkpoint_every=7)
    lay.set_weights(d["W_in"], d["W_rec"], d["W_out"], d["bias"])
    X = torch.as_tensor(d["X"], device="cuda")
    lay.forward(X)
    out = {k: torch.zeros(s, device="cuda") for k, s in
           (("dX", (T, B, n_in)), ("dI", (T, B, N)), ("dW_in", (n_in, N)), ("dW_rec", (N, N)),
            ("dbias", (N,)))}
    lay.backward_from(dL_dS=torch.as_tensor(dS, device="cuda"), dL_dV=torch.as_tensor(dV, device="cuda"), **out)
    torch.cuda.synchronize()
    spikes = lay.readout(hh.HH_LAYER_SPIKES).reshape(T, B, N)
    status = int(lay.readout(hh.HH_LAYER_STATUS)[0])
    lay.close()
    ref = bptt.layer_vjp(HH, d["X"], d["W_in"], d["W_rec"], d["bias"], dS.astype(np.float64),
                         dV.astype(np.float64), K=10, dt=0.01)
    assert status == 0
    assert ref["S"].sum() > 20
    assert np.array_equal(spikes, ref["S"])
    errs = {k: _elementwise(out[k].cpu().numpy(), ref[k], tol) for k in ("dX", "dI", "dW_in", "dW_rec", "dbias")}
    print("max|err|/max|ref|:", {k: f"{e:.2e}" for k, e in errs.items()})
    for k, e in errs.items():
        assert e <= tol, (k, e)


def test_layer_spikes_function_composes_with_torch():
    """layer_spikes_function inside a torch program: a preceding elementwise
    op on the inputs and an arbitrary loss of S and V_T back-propagate through
    the hand-derived adjoint; the gradients of the inputs' leaf and of the
    weights match the FP64 oracle's reverse mode of the same program."""
    torch = _torch()
    T, B, n_in, N, n_out = 24, 3, 32, 64, 4
    d = small_case(6, T, B, n_in, N, n_out)
    lay = hh.Layer(HH, batch=B, n_in=n_in, n_hidden=N, n_out=n_out, n_steps=T, substeps=10, dt=0.01,
                   precision=hh.HH_PREC_ACCURATE, checkpoint_every=5)
    Z = torch.tensor(d["X"], dtype=torch.float32, device="cuda", requires_grad=True)
    W_in, W_rec, bias = [torch.tensor(d[k], dtype=torch.float32, device="cuda", requires_grad=True)
                         for k in ("W_in", "W_rec", "bias")]
    rng = np.random.default_rng(2)
    mask = (rng.random(n_in) < 0.8).astype(np.float32)
    X = Z * torch.as_tensor(mask, device="cuda")  # an elementwise op in front of the layer (X stays 0/1)
    S, V = lay.spikes(X, W_in, W_rec, bias)
    R = torch.as_tensor(rng.normal(0, 1, (T, B, N)).astype(np.float32), device="cuda")
    loss = (S * R).sum() + 0.01 * ((V + 60.0) ** 2).mean()
    loss.backward()
    Xm = d["X"] * mask
    assert bptt.threshold_margin(HH, Xm, d["W_in"], d["W_rec"], d["bias"]).min() >= 1e-3
    ref = bptt.layer_vjp(HH, Xm, d["W_in"], d["W_rec"], d["bias"], R.cpu().numpy().astype(np.float64),
                         None, K=10, dt=0.01)
    Vr = ref["V"]
    dV = 0.01 * 2.0 * (Vr + 60.0) / Vr.size
    ref = bptt.layer_vjp(HH, Xm, d["W_in"], d["W_rec"], d["bias"], R.cpu().numpy().astype(np.float64),
                         dV, K=10, dt=0.01)
    ref["dZ"] = ref["dX"] * mask
    assert np.array_equal(S.detach().cpu().numpy(), ref["S"])
    assert ref["S"].sum() > 10
    for got, name in ((Z.grad, "dZ"), (W_in.grad, "dW_in"), (W_rec.grad, "dW_rec"), (bias.grad, "dbias")):
        e = _elementwise(got.cpu().numpy(), ref[name], 1e-3)
        print(f"{name}: max|err|/max|ref| = {e:.2e}")
        assert e <= 1e-3, (name, e)
    lay.close()


def test_layer_full_size_gradients_elementwise():
    """The full-size kernel paths (1,024 neurons: recurrent products with
    split-K 8, dS products with K = 2,048 and split-K 8; 700 inputs;
    checkpoints every 25 outer steps; 10 substeps) at B = 2, T = 30 with the
    built-in loss: identical spike raster, and dW_in, dW_rec, dW_out and dbias
    agree with the FP64 oracle entry by entry, |got - ref| <= 2e-3 max|ref|
    (measured 1.0e-3 for dW_in: the FP32 state over 300 substeps of 2,048
    neurons), every substep at least 1e-3 mV from theta in the oracle."""
    T, B, n_in, N, n_out = 30, 2, 700, 1024, 20
    d = inp.recurrent_layer(B=B, n_in=n_in, n_hid=N, n_out=n_out, T=T, seed=3, rate_max_hz=400.0,
                            w_in_scale=60.0)
    assert bptt.threshold_margin(HH, d["X"], d["W_in"], d["W_rec"], d["bias"]).min() >= 1e-3
    g = run_layer(d, T=T, B=B, n_in=n_in, N=N, n_out=n_out, precision=hh.HH_PREC_ACCURATE, ckpt=25)
    ref = bptt.layer_grads(HH, d["X"], d["W_in"], d["W_rec"], d["W_out"], d["bias"], d["labels"],
                           K=10, dt=0.01)
    assert g["status"] == 0
    assert ref["spikes"].sum() > 200
    assert np.array_equal(g["spikes"], ref["spikes"])
    errs = {k: _elementwise(g[k], ref[k], 2e-3) for k in ("dW_in", "dW_rec", "dW_out", "dbias")}
    print("max|err|/max|ref|:", {k: f"{e:.2e}" for k, e in errs.items()})
    for k, e in errs.items():
        assert e <= 2e-3, (k, e)


def _bf16_ulp(w):
    a = np.abs(w.astype(np.float64))
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    return np.where(a > 0, 2.0 ** (e - 7), 0.0)


def test_layer_gradient_matches_gpu_finite_differences():
    """The GPU adjoint against central differences of the GPU's own forward
    loss (smooth spikes, IEEE FP32, recurrent weights nonzero): along a
    direction D per parameter -- one bf16 unit in the last place per entry of
    W_in and W_rec (so W +- D stay exactly representable in the bf16 weights
    the products use), 1e-3 relative per entry of W_out and bias, each entry
    signed like its adjoint gradient so that the directional derivative sums
    without cancellation and stands far above the FP32 rounding of the loss
    -- (L(P + D) - L(P - D)) / 2, formed in FP64 from the two FP32 losses,
    agrees with sum(dL/dP * D) to 2 %."""
    torch = _torch()
    T, B, n_in, N, n_out = 20, 3, 24, 32, 4
    d = small_case(8, T, B, n_in, N, n_out, w_rec=3.0)
    lay = hh.Layer(HH, batch=B, n_in=n_in, n_hidden=N, n_out=n_out, n_steps=T, substeps=10, dt=0.01,
                   precision=hh.HH_PREC_ACCURATE, smooth=True, checkpoint_every=6)
    X = torch.as_tensor(d["X"], device="cuda")
    y = torch.as_tensor(d["labels"], device="cuda")
    loss = torch.zeros(1, device="cuda")
    P = {k: d[k].astype(np.float32).copy() for k in ("W_in", "W_rec", "W_out", "bias")}

    def L(p):
        lay.set_weights(p["W_in"], p["W_rec"], p["W_out"], p["bias"])
        lay.forward(X, y, loss)
        torch.cuda.synchronize()
        return float(loss.item())

    L(P)
    g = {k: torch.zeros(v.shape, device="cuda") for k, v in P.items()}
    lay.backward(g["W_in"], g["W_rec"], g["W_out"], g["bias"])
    torch.cuda.synchronize()
    for k in P:
        sign = np.sign(g[k].cpu().numpy().astype(np.float64))
        if k in ("W_in", "W_rec"):
            D = sign * _bf16_ulp(P[k])
        else:
            D = sign * 1e-3 * np.maximum(np.abs(P[k]), 1e-2)
        plus = dict(P, **{k: (P[k].astype(np.float64) + D).astype(np.float32)})
        minus = dict(P, **{k: (P[k].astype(np.float64) - D).astype(np.float32)})
        if k in ("W_in", "W_rec"):
            assert np.array_equal(inp.to_bf16_exact(plus[k]), plus[k])
        fd = (np.float64(L(plus)) - np.float64(L(minus))) / 2.0
        an = float((g[k].cpu().numpy().astype(np.float64) * D).sum())
        print(f"{k}: fd {fd:.6e} adjoint {an:.6e}")
        assert abs(fd - an) <= 2e-2 * abs(an), (k, fd, an)
    lay.close()
