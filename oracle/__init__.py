"""FP64 CPU oracle for the Hodgkin-Huxley hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA path: the C
source ``hh_oracle.c`` is compiled here with gcc into ``liboracle.so`` and
called through ctypes; the BPTT oracle (``oracle.bptt``) is plain PyTorch
CPU float64.

Parity pins: see ``tests/test_oracle_*.py`` (resting fixed point, spike
amplitude, repetitive-firing threshold, second-order convergence under dt
halving, removable singularities, Philox known-answer vectors, Poisson
moments, dense brute-force routing, central finite differences).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hh_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OR_MAX_CH = 8
OR_MAX_GATES = 12
_FORMS = {"const": 0, "exp": 1, "sigmoid": 2, "linoid": 3, "bell": 4}
_KINDS = {"ab": 0, "inftau": 1, "ca": 2}


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, -O2, no FP contraction, OpenMP)."""
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Fn(C.Structure):
    _fields_ = [("form", C.c_int32), ("pad", C.c_int32), ("a", C.c_double),
                ("vh", C.c_double), ("k", C.c_double), ("vh2", C.c_double),
                ("k2", C.c_double), ("c", C.c_double)]


class _Gate(C.Structure):
    _fields_ = [("kind", C.c_int32), ("power", C.c_int32), ("f1", _Fn), ("f2", _Fn)]


class _Channel(C.Structure):
    _fields_ = [("E", C.c_double), ("gbar", C.c_double), ("n_gates", C.c_int32),
                ("first_gate", C.c_int32)]


class _Model(C.Structure):
    _fields_ = [("C_m", C.c_double), ("n_channels", C.c_int32), ("n_gates", C.c_int32),
                ("ch", _Channel * OR_MAX_CH), ("g", _Gate * OR_MAX_GATES),
                ("ca_channel", C.c_int32), ("pad", C.c_int32), ("ca_tau", C.c_double),
                ("ca_k", C.c_double), ("ca_rest", C.c_double)]


def _p(a, ctype):
    return None if a is None else a.ctypes.data_as(C.POINTER(ctype))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            d, i32, i64, u64 = C.c_double, C.c_int32, C.c_int64, C.c_uint64
            P = C.POINTER
            L.or_rate.restype = d
            L.or_rate.argtypes = [P(_Fn), d]
            L.or_gate_inf_tau.argtypes = [P(_Gate), d, d, P(d), P(d)]
            L.or_init_neuron.argtypes = [P(_Model), d, P(d), P(d)]
            L.or_ionic_current.restype = d
            L.or_ionic_current.argtypes = [P(_Model), P(d), d, P(d)]
            L.or_step_neuron.restype = d
            L.or_step_neuron.argtypes = [P(_Model), P(d), d, d, d, d, d, d, i32, d, P(d), P(d)]
            L.or_simulate.restype = C.c_int
            L.or_simulate.argtypes = [P(_Model), i32, P(C.c_uint8), P(d), i64, i64, d, d, i32,
                                      P(d), P(d), P(d), P(d), P(i32), i32, P(i32), P(d), i32]
            L.or_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
            L.or_background_word.restype = C.c_uint32
            L.or_background_word.argtypes = [u64, i64, i64]
            L.or_poisson_table.restype = i32
            L.or_poisson_table.argtypes = [d, P(u64), i32]
            L.or_poisson_sample.restype = i32
            L.or_poisson_sample.argtypes = [C.c_uint32, P(u64), i32]
            L.or_background_lambda.restype = d
            L.or_background_normal.restype = d
            L.or_background_normal.argtypes = [u64, i64, i64]
            L.or_background_input.restype = d
            L.or_background_input.argtypes = [u64, i64, i64, P(u64), i32, d, d]
            L.or_background_lambda.argtypes = [i32, d, d]
            L.or_route.restype = C.c_int
            L.or_route.argtypes = [i64, i64, i32, P(i64), P(i32), P(d), P(C.c_uint8),
                                   P(i32), P(i32), i64, P(d), P(d)]
            L.or_simulate_network.restype = C.c_int
            L.or_simulate_network.argtypes = [
                P(_Model), i32, P(C.c_uint8), P(d), i64, i64, d, d, i32, P(d), P(d), P(d),
                P(i64), P(i32), P(d), P(C.c_uint8), d, d, d, d, i32, d, d, i32, d, u64, d, i32,
                P(i32), P(i32), i64, P(i64), i64, P(d), P(i32), i32, P(i32), P(d), i32]
            L.or_simulate_cable.restype = C.c_int
            L.or_simulate_cable.argtypes = [P(_Model), P(d), i64, P(i64), P(d), d, i64, d, d, P(d), P(d),
                                            P(d), P(d), P(i32), i32, P(i32), P(d)]
            L.or_sizeof_model.restype = i32
            L.or_sizeof_gate.restype = i32
            assert L.or_sizeof_model() == C.sizeof(_Model)
            assert L.or_sizeof_gate() == C.sizeof(_Gate)
            _lib = L
    return _lib


# ---------------------------------------------------------------------------
# marshalling of model tables (dicts from paper_2601_21407_gb300.inputs)
# ---------------------------------------------------------------------------

def _fn(t) -> _Fn:
    form, a, vh, k, vh2, k2, c = t
    return _Fn(_FORMS[form], 0, a, vh, k, vh2, k2, c)


def make_model(model: dict) -> _Model:
    M = _Model()
    M.C_m = model["C_m"]
    M.ca_channel = -1
    gi = 0
    for ci, ch in enumerate(model["channels"]):
        M.ch[ci].E = ch["E"]
        M.ch[ci].gbar = ch["gbar"]
        M.ch[ci].n_gates = len(ch["gates"])
        M.ch[ci].first_gate = gi
        for g in ch["gates"]:
            M.g[gi] = _Gate(_KINDS[g["kind"]], g["power"], _fn(g["f1"]), _fn(g["f2"]))
            gi += 1
    M.n_channels = len(model["channels"])
    M.n_gates = gi
    ca = model.get("calcium")
    if ca:
        names = [c["name"] for c in model["channels"]]
        M.ca_channel = names.index(ca["channel"])
        M.ca_tau, M.ca_k, M.ca_rest = ca["tau"], ca["k"], ca["rest"]
    return M


def _models_array(models):
    if isinstance(models, dict):
        models = [models]
    arr = (_Model * len(models))(*[make_model(m) for m in models])
    return arr, len(models)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Python API
# ---------------------------------------------------------------------------

def rate(fn_tuple, V: float) -> float:
    return lib().or_rate(C.byref(_fn(fn_tuple)), float(V))


def gate_inf_tau(gate: dict, V: float, Ca: float = 0.0):
    g = _Gate(_KINDS[gate["kind"]], gate["power"], _fn(gate["f1"]), _fn(gate["f2"]))
    inf, tau = C.c_double(), C.c_double()
    lib().or_gate_inf_tau(C.byref(g), float(V), float(Ca), C.byref(inf), C.byref(tau))
    return inf.value, tau.value


def init_neuron(model: dict, V0: float):
    M = make_model(model)
    p = np.zeros(OR_MAX_GATES)
    Ca = C.c_double()
    lib().or_init_neuron(C.byref(M), float(V0), _p(p, C.c_double), C.byref(Ca))
    return p[:M.n_gates].copy(), Ca.value


def ionic_current(model: dict, V: float, p, gbar=None) -> float:
    M = make_model(model)
    gb = np.array([c["gbar"] for c in model["channels"]] if gbar is None else gbar, dtype=np.float64)
    pp = np.zeros(OR_MAX_GATES)
    pp[:len(p)] = p
    return lib().or_ionic_current(C.byref(M), _p(gb, C.c_double), float(V), _p(pp, C.c_double))


def step_neuron(model: dict, V: float, p, Ca: float, dt: float, I: float,
                gE=0.0, EE=0.0, gI=0.0, EI=0.0, v_mode=0, gbar=None):
    M = make_model(model)
    gb = np.array([c["gbar"] for c in model["channels"]] if gbar is None else gbar, dtype=np.float64)
    pp = np.zeros(OR_MAX_GATES)
    pp[:len(p)] = p
    ca = C.c_double(Ca)
    Vn = lib().or_step_neuron(C.byref(M), _p(gb, C.c_double), dt, I, gE, EE, gI, EI, v_mode,
                              float(V), _p(pp, C.c_double), C.byref(ca))
    return Vn, pp[:M.n_gates].copy(), ca.value


def simulate(models, I, V0, T, dt, theta=0.0, v_mode=0, model_id=None, gbar=None,
             I_steps=None, trace=True, spk_cap=64, n_threads=0):
    """Independent neurons.  Returns dict(V [T][N] or None, counts [N],
    spk_step [N][cap], spk_frac [N][cap])."""
    marr, nm = _models_array(models)
    I = _f64(I)
    V0 = _f64(V0)
    N = V0.size
    gb = None
    if gbar is not None:
        g = np.asarray(gbar, dtype=np.float64)
        gb = np.zeros((OR_MAX_CH, N))
        gb[:g.shape[0]] = g
    mid = None if model_id is None else np.ascontiguousarray(model_id, dtype=np.uint8)
    Its = _f64(I_steps)
    Vt = np.empty((T, N)) if trace else None
    counts = np.zeros(N, dtype=np.int32)
    ss = np.full((N, spk_cap), -1, dtype=np.int32)
    sf = np.zeros((N, spk_cap))
    rc = lib().or_simulate(marr, nm, _p(mid, C.c_uint8), _p(gb, C.c_double), N, T, dt, theta,
                           v_mode, _p(I, C.c_double), _p(Its, C.c_double), _p(V0, C.c_double),
                           _p(Vt, C.c_double), _p(counts, C.c_int32), spk_cap,
                           _p(ss, C.c_int32), _p(sf, C.c_double), n_threads)
    if rc != 0:
        raise ValueError("or_simulate rejected its arguments")
    return {"V": Vt, "counts": counts, "spk_step": ss, "spk_frac": sf}


def sin_drive_steps(amp, freq_hz, phase, dt, T, t0=0):
    """The sinusoidal drive as per-step currents [T][N] in FP64:
    I(t) = amp sin(2 pi u(t) 2^-32) with the phase a 32-bit fraction of a
    cycle, u(t) = t F + P (mod 2^32), F = round(freq dt 2^32 / 1000),
    P = round(phase 2^32) mod 2^32 (integer arithmetic, so the phase is the
    same at any step count)."""
    amp = np.asarray(amp, dtype=np.float64)
    f = np.asarray(freq_hz, dtype=np.float32).astype(np.float64)
    ph = np.asarray(phase, dtype=np.float32).astype(np.float64)
    two32 = 4294967296.0
    F = np.mod(np.rint(f * dt * two32 / 1000.0), two32).astype(np.uint64)
    P = np.mod(np.rint(ph * two32), two32).astype(np.uint64)
    t = np.arange(t0, t0 + T, dtype=np.uint64)[:, None]
    u = (t * F[None, :] + P[None, :]) & np.uint64(0xFFFFFFFF)
    return np.asarray(amp, np.float32).astype(np.float64)[None, :] * np.sin(2.0 * np.pi * u.astype(np.float64) / two32)


def simulate_cable(model, parent, area, g_ax, I, V0, T, dt, theta=0.0, gbar=None, I_steps=None,
                   trace=True, spk_cap=64):
    """Multi-compartment neurons: compartments joined in a tree (parent[c], -1
    for a root) by the axial conductance g_ax (mS/cm^2 per unit area of the
    child), membrane areas `area` (relative), the cable term by the explicit
    second difference and the channels by exponential Euler.  Returns
    dict(V [T][N] or None, counts, spk_step, spk_frac)."""
    M = make_model(model)
    par = np.ascontiguousarray(parent, dtype=np.int64)
    N = par.size
    ar = _f64(area)
    gb = None
    if gbar is not None:
        g = np.asarray(gbar, dtype=np.float64)
        gb = np.zeros((OR_MAX_CH, N))
        gb[:g.shape[0]] = g
    Ic, V0d, Its = _f64(I), _f64(V0), _f64(I_steps)
    Vt = np.empty((T, N)) if trace else None
    counts = np.zeros(N, dtype=np.int32)
    ss = np.full((N, spk_cap), -1, dtype=np.int32)
    sf = np.zeros((N, spk_cap))
    rc = lib().or_simulate_cable(C.byref(M), _p(gb, C.c_double), N, _p(par, C.c_int64), _p(ar, C.c_double),
                                 float(g_ax), T, dt, theta, _p(Ic, C.c_double), _p(Its, C.c_double),
                                 _p(V0d, C.c_double), _p(Vt, C.c_double), _p(counts, C.c_int32), spk_cap,
                                 _p(ss, C.c_int32), _p(sf, C.c_double))
    if rc != 0:
        raise ValueError("or_simulate_cable rejected its arguments")
    return {"V": Vt, "counts": counts, "spk_step": ss, "spk_frac": sf}


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [o[i] for i in range(4)]


def background_word(seed, t, i):
    return lib().or_background_word(int(seed), int(t), int(i))


def poisson_table(lam, cap=64):
    thr = np.zeros(cap, dtype=np.uint64)
    n = lib().or_poisson_table(float(lam), _p(thr, C.c_uint64), cap)
    return thr[:n].copy()


def poisson_sample(u, thr):
    thr = np.ascontiguousarray(thr, dtype=np.uint64)
    return lib().or_poisson_sample(int(u), _p(thr, C.c_uint64), thr.size)


def background_normal(seed, t, i):
    return lib().or_background_normal(C.c_uint64(seed), int(t), int(i))


def background_input(seed, t, i, K, rate_hz, dt, w, sd=0.0):
    """The network oracle's background input of neuron i at step t (the
    same C function its loop calls)."""
    thr = poisson_table(background_lambda(K, rate_hz, dt))
    tt = (C.c_uint64 * len(thr))(*[int(x) for x in thr])
    return lib().or_background_input(C.c_uint64(seed), int(t), int(i), tt, len(thr), float(w), float(sd))


def background_lambda(K, rate_hz, dt_ms):
    return lib().or_background_lambda(int(K), float(rate_hz), float(dt_ms))


def route(N, T, D, row_ptr, col, w, inh, spk_step, spk_idx):
    """Open-loop routing: delivered sums [T][N] for excitatory and inhibitory
    presynaptic neurons (float64)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    ww = _f64(w)
    ih = np.ascontiguousarray(inh, dtype=np.uint8)
    ss = np.ascontiguousarray(spk_step, dtype=np.int32)
    si = np.ascontiguousarray(spk_idx, dtype=np.int32)
    sE = np.zeros((T, N))
    sI = np.zeros((T, N))
    rc = lib().or_route(N, T, D, _p(rp, C.c_int64), _p(cl, C.c_int32), _p(ww, C.c_double),
                        _p(ih, C.c_uint8), _p(ss, C.c_int32), _p(si, C.c_int32), ss.size,
                        _p(sE, C.c_double), _p(sI, C.c_double))
    if rc != 0:
        raise ValueError("or_route rejected its arguments")
    return sE, sI


def simulate_network(models, net, T, dt, D, syn, bg=None, I=None, theta=0.0, v_mode=0,
                     model_id=None, gbar=None, forced=None, trace_idx=None, spk_cap=256,
                     n_threads=0, seed=0, I_steps=None, syn_current=False):
    """Network of point neurons.  net: dict(row_ptr, col, w, inh, V0);
    syn: dict(tau_E, tau_I, E_E, E_I, area_cm2); bg: dict(rate_hz, K, w[, sd])
    or None (sd > 0: compound background, the sum of the count's Gaussian
    amplitudes); forced: (steps, idx) spike list for open-loop routing, or
    None.  syn_current: synapses inject their filtered current (weights in
    uA/cm^2, excitatory minus inhibitory) instead of a conductance."""
    marr, nm = _models_array(models)
    V0 = _f64(net["V0"])
    N = V0.size
    rp = np.ascontiguousarray(net["row_ptr"], dtype=np.int64)
    cl = np.ascontiguousarray(net["col"], dtype=np.int32)
    ww = _f64(net["w"])
    ih = np.ascontiguousarray(net["inh"], dtype=np.uint8)
    gb = None
    if gbar is not None:
        g = np.asarray(gbar, dtype=np.float64)
        gb = np.zeros((OR_MAX_CH, N))
        gb[:g.shape[0]] = g
    mid = None if model_id is None else np.ascontiguousarray(model_id, dtype=np.uint8)
    Ic = _f64(I)
    Its = _f64(I_steps)
    if Its is not None and Its.shape != (T, N):
        raise ValueError("I_steps must be [T][N]")
    if forced is not None:
        fs = np.ascontiguousarray(forced[0], dtype=np.int32)
        fi = np.ascontiguousarray(forced[1], dtype=np.int32)
        nf = fs.size
    else:
        fs = fi = None
        nf = -1
    tix = None if trace_idx is None else np.ascontiguousarray(trace_idx, dtype=np.int64)
    ntr = 0 if tix is None else tix.size
    Vt = np.empty((T, ntr)) if ntr else None
    counts = np.zeros(N, dtype=np.int32)
    ss = np.full((N, spk_cap), -1, dtype=np.int32)
    sf = np.zeros((N, spk_cap))
    bg = bg or {"rate_hz": 0.0, "K": 0, "w": 0.0}
    rc = lib().or_simulate_network(
        marr, nm, _p(mid, C.c_uint8), _p(gb, C.c_double), N, T, dt, theta, v_mode,
        _p(Ic, C.c_double), _p(Its, C.c_double), _p(V0, C.c_double), _p(rp, C.c_int64), _p(cl, C.c_int32),
        _p(ww, C.c_double), _p(ih, C.c_uint8), syn["tau_E"], syn["tau_I"], syn["E_E"],
        syn["E_I"], D, syn["area_cm2"], bg["rate_hz"], bg["K"], bg["w"], seed, float(bg.get("sd", 0.0)),
        1 if syn_current else 0,
        _p(fs, C.c_int32), _p(fi, C.c_int32), nf, _p(tix, C.c_int64), ntr,
        _p(Vt, C.c_double), _p(counts, C.c_int32), spk_cap, _p(ss, C.c_int32),
        _p(sf, C.c_double), n_threads)
    if rc != 0:
        raise ValueError("or_simulate_network rejected its arguments")
    return {"V": Vt, "counts": counts, "spk_step": ss, "spk_frac": sf}
