"""FP64 oracle of the differentiable recurrent HH layer (test infrastructure).

Plain PyTorch CPU float64; the reverse mode is torch autograd, so the
gradients are those of the forward program as written here.  Only tests,
the smoke check and the benchmark's CPU-baseline leg may use it.

Forward (per sample; Methods, Eq. hh_eq_full with the exponential-Euler
discretisation; input current "generated by the parameters of the former
layers", Methods "Analysis of C_m"):
    I_t     = bias + X_t W_in + S_{t-1} W_rec                (S_{-1} = 0)
    for k = 1..K substeps of dt (I_t held):
        gates  p <- p + (p_inf(V) - p)(1 - exp(-dt (alpha + beta)))
        V      <- V + (I_t - I_ion)/G (1 - exp(-dt G / C_m))
        c_{t,k} = H(V_k - theta) (1 - H(V_{k-1} - theta))
    S_t     = sum_k c_{t,k}          (an upward crossing in the outer step)
    r       = (1/T) sum_t S_t,   logits = r W_out^T,   loss = mean_b CE(logits_b, y_b)
Spike surrogate: the forward is the Heaviside step; the backward replaces
dH(x)/dx by 1/(1 + beta |x|)^2 (beta in 1/mV) and treats the
(1 - H(V_{k-1} - theta)) factor as a constant.  With smooth=True the step is
replaced in the forward as well by the smooth step
    sigma(x) = 0.5 + 0.5 beta x / (1 + beta |x|)
(and the (1 - H) factor by 1 - sigma(V_{k-1} - theta)): a differentiable
program on which central finite differences pin the reverse mode.
"""
from __future__ import annotations

import torch

DT = torch.float64


def _rate(fn, V):
    form, a, vh, k, vh2, k2, c = fn
    if form == "const":
        r = torch.full_like(V, a)
    elif form == "exp":
        r = a * torch.exp((V - vh) / k)
    elif form == "sigmoid":
        r = a / (1.0 + torch.exp((V - vh) / k))
    elif form == "linoid":
        x = V - vh
        y = x / k
        small = y.abs() < 1e-6
        ys = torch.where(small, torch.ones_like(y), y)
        full = a * k * ys / (-torch.expm1(-ys))
        series = a * k * (1.0 + 0.5 * y + y * y / 12.0)
        r = torch.where(small, series, full)
    else:  # bell
        r = a / (torch.exp((V - vh) / k) + torch.exp((V - vh2) / k2))
    return r + c


def _gates(model):
    return [g for ch in model["channels"] for g in ch["gates"]]


def init_state(model, V0):
    """Gates at steady state p_inf(V0) (alpha/beta gates)."""
    ps = []
    for g in _gates(model):
        al, be = _rate(g["f1"], V0), _rate(g["f2"], V0)
        ps.append(al / (al + be))
    return ps


def substep(model, V, ps, I, dt):
    """One exponential-Euler step of the point neuron (current input)."""
    new = []
    for g, p in zip(_gates(model), ps):
        al, be = _rate(g["f1"], V), _rate(g["f2"], V)
        s = al + be
        inf = al / s
        new.append(p + (inf - p) * (-torch.expm1(-dt * s)))
    G = torch.zeros_like(V)
    Iion = torch.zeros_like(V)
    q = 0
    for ch in model["channels"]:
        eta = torch.ones_like(V)
        for g in ch["gates"]:
            eta = eta * new[q] ** g["power"]
            q += 1
        gx = ch["gbar"] * eta
        G = G + gx
        Iion = Iion + gx * (V - ch["E"])
    Vn = V + (I - Iion) / G * (-torch.expm1(-dt * G / model["C_m"]))
    return Vn, new


class _Spike(torch.autograd.Function):
    """Heaviside forward, 1/(1+beta|x|)^2 backward."""

    @staticmethod
    def forward(ctx, x, beta):
        ctx.save_for_backward(x)
        ctx.beta = beta
        return (x >= 0).to(x.dtype)

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        return g / (1.0 + ctx.beta * x.abs()) ** 2, None


def _smooth(x, beta):
    return 0.5 + 0.5 * beta * x / (1.0 + beta * x.abs())


def layer_run(model, X, W_in, W_rec, bias, *, dt=0.01, K=10, theta=0.0, beta=0.5, smooth=False,
              V0=-65.0, currents=None):
    """The layer's outputs as a differentiable program of its inputs and
    weights: X [T, B, n_in], W_in [n_in, N], W_rec [N, N], bias [N].
    Returns (S [T, B, N], V_T [B, N]); if `currents` is a list, the input
    current I_t of every outer step is appended to it (with retain_grad)."""
    T, B, _ = X.shape
    N = W_in.shape[1]
    V = torch.full((B, N), float(V0), dtype=DT)
    ps = init_state(model, V)
    S_prev = torch.zeros((B, N), dtype=DT)
    spikes = []
    for t in range(T):
        I = bias + X[t] @ W_in + S_prev @ W_rec
        if currents is not None:
            if I.requires_grad:
                I.retain_grad()
            currents.append(I)
        s_t = torch.zeros((B, N), dtype=DT)
        for _ in range(K):
            Vn, ps = substep(model, V, ps, I, dt)
            if smooth:
                c = _smooth(Vn - theta, beta) * (1.0 - _smooth(V - theta, beta))
            else:
                c = _Spike.apply(Vn - theta, beta) * (1.0 - (V >= theta).to(DT)).detach()
            s_t = s_t + c
            V = Vn
        spikes.append(s_t)
        S_prev = s_t
    return torch.stack(spikes), V


def threshold_margin(model, X, W_in, W_rec, bias, *, dt=0.01, K=10, theta=0.0, V0=-65.0):
    """min over every substep of |V_k - theta| per (sample, neuron), [B, N],
    from the FP64 forward.  The surrogate gradient switches where V_{k-1}
    crosses theta (the (1 - H(V_{k-1} - theta)) factor), so a trajectory that
    passes closer to theta than another arithmetic's rounding of V can put a
    crossing in a different substep and change the gradient by O(1): this is
    the conditioning of the method's gradient, read off the oracle alone."""
    with torch.no_grad():
        X, W_in, W_rec, bias = (torch.as_tensor(a, dtype=DT) for a in (X, W_in, W_rec, bias))
        T, B, _ = X.shape
        N = W_in.shape[1]
        V = torch.full((B, N), float(V0), dtype=DT)
        ps = init_state(model, V)
        S_prev = torch.zeros((B, N), dtype=DT)
        m = torch.full((B, N), float("inf"), dtype=DT)
        for t in range(T):
            I = bias + X[t] @ W_in + S_prev @ W_rec
            s_t = torch.zeros((B, N), dtype=DT)
            for _ in range(K):
                Vn, ps = substep(model, V, ps, I, dt)
                m = torch.minimum(m, (Vn - theta).abs())
                s_t = s_t + ((Vn >= theta) & ~(V >= theta)).to(DT)
                V = Vn
            S_prev = s_t
    return m.numpy()


def layer_forward(model, X, W_in, W_rec, W_out, bias, labels, *, dt=0.01, K=10, theta=0.0,
                  beta=0.5, smooth=False, V0=-65.0, return_all=False):
    """X: [T, B, n_in] (0/1), W_in [n_in, N], W_rec [N, N], W_out [n_out, N],
    bias [N], labels [B] (long).  Returns loss (and optionally spikes,
    logits, final V)."""
    S, V = layer_run(model, X, W_in, W_rec, bias, dt=dt, K=K, theta=theta, beta=beta, smooth=smooth, V0=V0)
    r = S.sum(0) / S.shape[0]
    logits = r @ W_out.T
    loss = torch.nn.functional.cross_entropy(logits, labels)
    if return_all:
        return loss, {"spikes": S, "logits": logits, "V": V}
    return loss


def layer_vjp(model, X, W_in, W_rec, bias, dS, dV, **kw):
    """Gradients of L = sum(dS * S) + sum(dV * V_T) with respect to X, W_in,
    W_rec, bias and every outer step's input current I_t (float64 numpy
    arrays; dS [T, B, N] and dV [B, N] may be None)."""
    leaves = [torch.tensor(a, dtype=DT, requires_grad=True) for a in (X, W_in, W_rec, bias)]
    cur = []
    S, V = layer_run(model, *leaves, currents=cur, **kw)
    L = torch.zeros((), dtype=DT)
    if dS is not None:
        L = L + (S * torch.tensor(dS, dtype=DT)).sum()
    if dV is not None:
        L = L + (V * torch.tensor(dV, dtype=DT)).sum()
    L.backward()
    out = {"S": S.detach().numpy(), "V": V.detach().numpy(), "dI": torch.stack([c.grad for c in cur]).numpy()}
    for name, p in zip(("X", "W_in", "W_rec", "bias"), leaves):
        out["d" + name] = p.grad.numpy()
    return out


def layer_grads(model, X, W_in, W_rec, W_out, bias, labels, **kw):
    """Loss and gradients w.r.t. (W_in, W_rec, W_out, bias) in float64."""
    params = [torch.tensor(p, dtype=DT, requires_grad=True) for p in (W_in, W_rec, W_out, bias)]
    Xt = torch.tensor(X, dtype=DT)
    y = torch.tensor(labels, dtype=torch.long)
    loss, aux = layer_forward(model, Xt, *params, y, return_all=True, **kw)
    loss.backward()
    out = {"loss": float(loss.detach()), "spikes": aux["spikes"].detach().numpy(),
           "logits": aux["logits"].detach().numpy(), "V": aux["V"].detach().numpy()}
    for name, p in zip(("W_in", "W_rec", "W_out", "bias"), params):
        out["d" + name] = p.grad.numpy()
    return out


def layer_loss(model, X, W_in, W_rec, W_out, bias, labels, **kw):
    with torch.no_grad():
        return float(layer_forward(model, torch.tensor(X, dtype=DT), torch.tensor(W_in, dtype=DT),
                                   torch.tensor(W_rec, dtype=DT), torch.tensor(W_out, dtype=DT),
                                   torch.tensor(bias, dtype=DT), torch.tensor(labels, dtype=torch.long),
                                   **kw))
