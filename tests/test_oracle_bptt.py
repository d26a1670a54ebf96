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


@pytest.mark.parametrize("beta", [0.5, 2.0])
def test_surrogate_derivative_of_one_substep(beta):
    """The Heaviside program's spike gradient is the stated surrogate
    1/(1 + beta |x|)^2, x = V_1 - theta (the reading of the silent spike
    derivative): one neuron, one outer step of one substep from V_0 = -65 mV
    below theta, so S = H(V_1 - theta) and dL/dbias = dL/dS * sur(x) * dV_1/dI.
    dV_1/dI comes from a central difference of the forward (V_1 is smooth in
    I), dL/dS from the two-class cross-entropy written out here, and the
    threshold is placed at x = -3 .. +2 mV below and above V_1; a wrong
    exponent, a misplaced beta or a dropped |.| changes the ratio."""
    dt, b0, w = 0.01, 500.0, 1.5
    X = np.ones((1, 1, 1))
    W_in = np.zeros((1, 1))
    W_rec = np.zeros((1, 1))
    W_out = np.array([[w], [0.0]])
    y = np.array([1])

    def V1(bias, theta=0.0):
        return bptt.layer_grads(HH, X, W_in, W_rec, W_out, np.array([bias]), y, K=1, dt=dt,
                                theta=theta, beta=beta)["V"][0, 0]

    v1 = V1(b0)
    assert -65.0 < v1 - 3.0  # theta stays above V_0 for every x below
    h = 1e-3
    dVdI = (V1(b0 + h) - V1(b0 - h)) / (2 * h)
    assert 0.0 < dVdI < dt  # dV/dI = (1 - e^{-dt G/C})/G < dt/C
    for x in (-3.0, -0.5, 0.25, 2.0):
        theta = v1 - x
        g = bptt.layer_grads(HH, X, W_in, W_rec, W_out, np.array([b0]), y, K=1, dt=dt, theta=theta,
                             beta=beta)
        S = g["spikes"][0, 0, 0]
        assert S == (1.0 if x >= 0 else 0.0)
        # L = log(1 + e^{w S}) (label 1, logits (w S, 0)); dL/dS = w e^{wS}/(1 + e^{wS})
        dLdS = w * np.exp(w * S) / (1.0 + np.exp(w * S))
        ratio = g["dbias"][0] / (dLdS * dVdI)
        assert abs(ratio - 1.0 / (1.0 + beta * abs(x)) ** 2) <= 1e-6, (x, ratio)
        assert abs(g["dW_in"][0, 0] - g["dbias"][0]) <= 1e-15


def test_vjp_of_spike_and_voltage_outputs():
    """layer_vjp (gradients of <dS, S> + <dV, V_T>, the cotangents a larger
    model hands the layer): on the smooth-spike program every sampled entry of
    dX, dW_rec and dbias matches a central difference to 1e-5, and the input
    current's gradient ties them together as the linear map I_t = bias +
    X_t W_in + S_{t-1} W_rec requires (dbias = sum dI, dX_t = dI_t W_in^T,
    dW_in = sum_t X_t^T dI_t)."""
    X, W_in, W_rec, W_out, bias, y = _small(seed=5)
    X = X * 0.7 + 0.1  # real-valued inputs (a preceding layer's output)
    rng = np.random.default_rng(7)
    T, B, N = X.shape[0], X.shape[1], W_in.shape[1]
    dS = rng.normal(0, 1.0, (T, B, N))
    dV = rng.normal(0, 0.05, (B, N))
    kw = dict(K=4, dt=0.02, smooth=True)
    g = bptt.layer_vjp(HH, X, W_in, W_rec, bias, dS, dV, **kw)
    assert np.allclose(g["dbias"], g["dI"].sum((0, 1)), rtol=1e-12, atol=1e-14)
    assert np.allclose(g["dX"], g["dI"] @ W_in.T, rtol=1e-12, atol=1e-14)
    assert np.allclose(g["dW_in"], np.einsum("tbi,tbn->in", X, g["dI"]), rtol=1e-12, atol=1e-14)

    def L(Xa, Wr, b):
        import torch
        with torch.no_grad():
            S, V = bptt.layer_run(HH, *(torch.tensor(a, dtype=torch.float64) for a in (Xa, W_in, Wr, b)), **kw)
        return float((S.numpy() * dS).sum() + (V.numpy() * dV).sum())

    for name, P in (("X", X), ("W_rec", W_rec), ("bias", bias)):
        flat = P.reshape(-1)
        for j in rng.choice(flat.size, size=min(5, flat.size), replace=False):
            h = 1e-5 * max(1.0, abs(flat[j]))
            old = flat[j]
            flat[j] = old + h
            lp = L(X, W_rec, bias)
            flat[j] = old - h
            lm = L(X, W_rec, bias)
            flat[j] = old
            fd = (lp - lm) / (2 * h)
            an = g["d" + name].reshape(-1)[j]
            assert abs(fd - an) <= 1e-5 * max(1e-3, abs(fd), abs(an)), (name, j, fd, an)
