"""Pins of the FP64 BPTT oracle (recurrent HH layer): central finite
differences of the smooth-spike program, reduction to independent neurons
checked against the C oracle, and the closed-form readout gradient."""
import numpy as np
import pytest

import oracle
from oracle import bptt
from paper_2601_21407_gb300 import inputs as inp

HH = inp.CLASSIC_HH


def _small(seed=0, B=2, N=6, T=6, n_in=5):
    rng = np.random.default_rng(seed)
    X = (rng.random((T, B, n_in)) < 0.3).astype(np.float64)
    W_in = rng.normal(0, 6.0, (n_in, N))
    W_rec = rng.normal(0, 3.0, (N, N))
    W_out = rng.normal(0, 1.0, (3, N))
    bias = rng.uniform(4, 12, N)
    y = rng.integers(0, 3, B)
    return X, W_in, W_rec, W_out, bias, y


def test_reverse_mode_matches_central_differences():
    """Smooth-spike program: every gradient entry of W_in, W_rec, W_out and
    bias agrees with a central difference (h = 1e-5 relative) to 1e-5."""
    X, W_in, W_rec, W_out, bias, y = _small()
    kw = dict(K=4, dt=0.02, smooth=True)
    g = bptt.layer_grads(HH, X, W_in, W_rec, W_out, bias, y, **kw)
    params = {"W_in": W_in, "W_rec": W_rec, "W_out": W_out, "bias": bias}
    rng = np.random.default_rng(1)
    for name, P in params.items():
        flat = P.reshape(-1)
        for j in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            h = 1e-5 * max(1.0, abs(flat[j]))
            old = flat[j]
            flat[j] = old + h
            lp = bptt.layer_loss(HH, X, W_in, W_rec, W_out, bias, y, **kw)
            flat[j] = old - h
            lm = bptt.layer_loss(HH, X, W_in, W_rec, W_out, bias, y, **kw)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            an = g["d" + name].reshape(-1)[j]
            assert abs(fd - an) <= 1e-5 * max(1e-3, abs(fd), abs(an)), (name, j, fd, an)


def test_reduces_to_independent_neurons():
    """With W_in = W_rec = 0 each hidden neuron is a classic HH neuron driven by
    its bias: the layer's spike raster equals the C oracle's threshold
    crossings (outer step = 10 substeps) and V matches to 1e-9 mV."""
    T, K, dt, N = 60, 10, 0.01, 8
    bias = np.linspace(2.0, 16.0, N)
    X = np.zeros((T, 1, 3))
    g = bptt.layer_grads(HH, X, np.zeros((3, N)), np.zeros((N, N)), np.zeros((2, N)), bias,
                         np.array([0]), K=K, dt=dt)
    ref = oracle.simulate(HH, bias, np.full(N, -65.0), T * K, dt)
    assert np.abs(g["V"][0] - ref["V"][-1]).max() < 1e-9
    for i in range(N):
        outer = sorted(set(int(s) // K for s in ref["spk_step"][i][: ref["counts"][i]]))
        got = np.nonzero(g["spikes"][:, 0, i])[0].tolist()
        assert got == outer
    assert g["spikes"].sum() > 5


def test_readout_gradient_closed_form():
    """dL/dW_out = (softmax(logits) - onehot(y))^T r / B with r the mean spike
    count, in the surrogate (Heaviside) program."""
    X, W_in, W_rec, W_out, bias, y = _small(seed=3, B=3, N=7, T=20)
    g = bptt.layer_grads(HH, X, W_in, W_rec, W_out, bias, y, K=10, dt=0.01)
    r = g["spikes"].mean(0)
    lg = r @ W_out.T
    p = np.exp(lg - lg.max(1, keepdims=True))
    p /= p.sum(1, keepdims=True)
    p[np.arange(len(y)), y] -= 1.0
    dW = p.T @ r / len(y)
    assert np.allclose(g["dW_out"], dW, rtol=1e-12, atol=1e-14)
    assert np.allclose(g["logits"], lg, rtol=1e-12)
    assert g["spikes"].sum() > 0
