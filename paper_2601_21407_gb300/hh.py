"""Thin ctypes binding of libhh (include/hh.h).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of libhh.so.  The functions keep the C names (hh_create_network,
hh_set_channels, hh_step_n, hh_reset, hh_route_spikes, hh_readout,
hh_destroy, hh_last_error); ``Network`` is a small convenience wrapper that
owns a handle and passes torch device tensors' data pointers.

There is no CPU fallback: if libhh.so cannot be built or loaded, ``lib()``
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None

HH_OK, HH_EINVAL, HH_ENOMEM, HH_ECUDA, HH_ETIMEOUT, HH_ESTATE, HH_EUNSUPPORTED, HH_EOVERFLOW = range(8)
HH_FN = {"const": 0, "exp": 1, "sigmoid": 2, "linoid": 3, "bell": 4}
HH_GATE = {"ab": 0, "inftau": 1, "ca": 2}
HH_MAX_CHANNELS, HH_MAX_GATES_PER_CHANNEL, HH_MAX_GATES, HH_MAX_MODELS = 8, 3, 8, 4
HH_PREC_FAST, HH_PREC_ACCURATE, HH_PREC_COMPENSATED, HH_PREC_POLY = 0, 1, 2, 3
HH_POLY_V_LO, HH_POLY_V_HI, HH_POLY_REL_ERR = -120.0, 80.0, 5e-7
HH_V_EXP_EULER, HH_V_FWD_EULER = 0, 1
HH_KERNELS_SPECIALISED, HH_KERNELS_TABLE, HH_KERNELS_PERSISTENT = 0, 1, 2
(HH_READ_V, HH_READ_GATES, HH_READ_CA, HH_READ_G_SYN, HH_READ_STATUS, HH_READ_TIME,
 HH_READ_N_OUT, HH_READ_PROFILE, HH_READ_SURROGATE, HH_READ_POLY) = range(10)
HH_KERNEL_NEURON, HH_KERNEL_ROUTE, HH_KERNEL_COUNT = 0, 1, 2
HH_STATUS_SPIKE_OVERFLOW, HH_STATUS_NONFINITE, HH_STATUS_BARRIER_TIMEOUT = 1, 2, 4


class HHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hh status {status}: {msg}")
        self.status = status


class hh_fn(C.Structure):
    _fields_ = [("form", C.c_int32), ("a", C.c_float), ("vh", C.c_float), ("k", C.c_float),
                ("vh2", C.c_float), ("k2", C.c_float), ("c", C.c_float)]


class hh_gate(C.Structure):
    _fields_ = [("kind", C.c_int32), ("power", C.c_int32), ("f1", hh_fn), ("f2", hh_fn)]


class hh_channel(C.Structure):
    _fields_ = [("E_rev", C.c_float), ("gbar", C.c_float), ("n_gates", C.c_int32),
                ("gates", hh_gate * HH_MAX_GATES_PER_CHANNEL)]


class hh_model_desc(C.Structure):
    _fields_ = [("C_m", C.c_float), ("n_channels", C.c_int32),
                ("channels", hh_channel * HH_MAX_CHANNELS), ("ca_channel", C.c_int32),
                ("ca_tau", C.c_float), ("ca_k", C.c_float), ("ca_rest", C.c_float)]


class hh_morphology(C.Structure):
    _fields_ = [("n_dendrites", C.c_int32), ("n_per_dendrite", C.c_int32), ("g_axial", C.c_float),
                ("soma_area_ratio", C.c_float)]


HH_CABLE_LANES = 32


class hh_net_desc(C.Structure):
    _fields_ = [("n_neurons", C.c_int64), ("n_nets", C.c_int32), ("net_offsets", C.c_void_p),
                ("dt_ms", C.c_double), ("v_threshold", C.c_float), ("v_update", C.c_int32),
                ("precision", C.c_int32), ("kernels", C.c_int32), ("V0", C.c_void_p),
                ("I_const", C.c_void_p),
                ("model_id", C.c_void_p), ("n_synapses", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("weight", C.c_void_p), ("is_inhibitory", C.c_void_p),
                ("tau_E", C.c_float), ("tau_I", C.c_float), ("E_E", C.c_float),
                ("E_I", C.c_float), ("delay_steps", C.c_int32), ("area_cm2", C.c_float),
                ("bg_rate_hz", C.c_float), ("bg_sources", C.c_int32), ("bg_weight_nS", C.c_float),
                ("seed", C.c_uint64), ("stream", C.c_void_p), ("sin_amp", C.c_void_p),
                ("sin_freq_hz", C.c_void_p), ("sin_phase", C.c_void_p), ("morph", C.POINTER(hh_morphology)),
                ("syn_mode", C.c_int32), ("bg_weight_sd", C.c_float)]


HH_SYN_CONDUCTANCE, HH_SYN_CURRENT = 0, 1


class hh_spike(C.Structure):
    _fields_ = [("step", C.c_int32), ("neuron", C.c_int32), ("frac", C.c_float)]


class hh_neurons_noalloc(C.Structure):
    _fields_ = [("n_neurons", C.c_int64), ("dt_ms", C.c_double), ("v_threshold", C.c_float),
                ("v_update", C.c_int32), ("precision", C.c_int32), ("V", C.c_void_p),
                ("V_lo", C.c_void_p), ("gates", C.c_void_p), ("gates_lo", C.c_void_p),
                ("Ca", C.c_void_p), ("I_const", C.c_void_p), ("gbar", C.c_void_p),
                ("status", C.c_void_p), ("init_state", C.c_int32), ("stream", C.c_void_p)]


HH_NOALLOC_MAX_NEURONS = 1 << 20


class hh_surrogate_desc(C.Structure):
    _fields_ = [("window", C.c_int32), ("v_envelope", C.c_float), ("train_neurons", C.c_int32),
                ("train_windows", C.c_int32), ("epochs", C.c_int32), ("batch", C.c_int32),
                ("lr", C.c_float), ("seed", C.c_uint64), ("I_min", C.c_float), ("I_max", C.c_float),
                ("gbar_sigma", C.c_float), ("V0_min", C.c_float), ("V0_max", C.c_float),
                ("err_V", C.c_float), ("err_p", C.c_float)]


class hh_surrogate_report(C.Structure):
    _fields_ = [("train_windows", C.c_int64), ("train_loss", C.c_float), ("val_loss", C.c_float),
                ("out_scale_V", C.c_float)]


class hh_layer_desc(C.Structure):
    _fields_ = [("batch", C.c_int32), ("n_in", C.c_int32), ("n_hidden", C.c_int32),
                ("n_out", C.c_int32), ("n_steps", C.c_int32), ("substeps", C.c_int32),
                ("dt_ms", C.c_double), ("v_threshold", C.c_float), ("v_init", C.c_float),
                ("surrogate_beta", C.c_float), ("precision", C.c_int32), ("smooth", C.c_int32),
                ("checkpoint_every", C.c_int32), ("stream", C.c_void_p)]


class hh_grads(C.Structure):
    _fields_ = [("dW_in", C.c_void_p), ("dW_rec", C.c_void_p), ("dW_out", C.c_void_p),
                ("dbias", C.c_void_p), ("dI", C.c_void_p), ("dX", C.c_void_p)]


HH_LAYER_SPIKES, HH_LAYER_V, HH_LAYER_STATUS = 0, 1, 2


class hh_kernel_time(C.Structure):
    _fields_ = [("launches", C.c_int64), ("total_ms", C.c_double)]


class hh_peaks(C.Structure):
    _fields_ = [("ffma_per_s", C.c_double), ("ex2_per_s", C.c_double), ("rcp_per_s", C.c_double)]


HH_TUNE_MAX = 16


class hh_tune_report(C.Structure):
    _fields_ = [("n", C.c_int32), ("best", C.c_int32), ("neuron_block", C.c_int32 * HH_TUNE_MAX),
                ("route_blocks", C.c_int32 * HH_TUNE_MAX), ("ms", C.c_float * HH_TUNE_MAX)]


class hh_record(C.Structure):
    _fields_ = [("V_trace", C.c_void_p), ("trace_idx", C.c_void_p), ("n_trace", C.c_int32),
                ("spikes", C.c_void_p), ("spike_cap", C.c_int64), ("n_spikes", C.c_void_p),
                ("counts", C.c_void_p)]


EXPORTS = ["hh_create_network", "hh_set_channels", "hh_step_n", "hh_reset", "hh_route_spikes",
           "hh_readout", "hh_profile", "hh_step_neurons_noalloc", "hh_gemm_bf16", "hh_destroy",
           "hh_last_error", "hh_version", "hh_layer_create", "hh_layer_set_weights",
           "hh_layer_forward", "hh_backward", "hh_backward_from", "hh_layer_readout", "hh_layer_destroy",
           "hh_surrogate_train", "hh_surrogate_enable", "hh_measure_peaks", "hh_set_wait_limits",
           "hh_poly_fit", "hh_set_route_pull", "hh_state_size", "hh_save_state", "hh_load_state",
           "hh_set_launch_shape", "hh_autotune"]


def lib_path() -> str:
    return os.path.join(_HERE, "libhh.so")


def lib():
    """Build (if stale) and load libhh.so.  Raises when it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            from . import _build
            _build.build()
            L = C.CDLL(lib_path())
            P = C.POINTER
            vp = C.c_void_p
            L.hh_create_network.restype = C.c_int
            L.hh_create_network.argtypes = [P(hh_net_desc), P(vp)]
            L.hh_set_channels.restype = C.c_int
            L.hh_set_channels.argtypes = [vp, C.c_int32, P(hh_model_desc), vp]
            L.hh_step_n.restype = C.c_int
            L.hh_step_n.argtypes = [vp, C.c_int32, vp, P(hh_record)]
            L.hh_reset.restype = C.c_int
            L.hh_reset.argtypes = [vp, vp]
            L.hh_route_spikes.restype = C.c_int
            L.hh_route_spikes.argtypes = [vp, vp, vp, C.c_int64, C.c_int32, vp, vp]
            L.hh_readout.restype = C.c_int
            L.hh_readout.argtypes = [vp, C.c_int32, vp, C.c_size_t, P(C.c_size_t)]
            L.hh_profile.restype = C.c_int
            L.hh_profile.argtypes = [vp, C.c_int32]
            L.hh_step_neurons_noalloc.restype = C.c_int
            L.hh_step_neurons_noalloc.argtypes = [P(hh_model_desc), P(hh_neurons_noalloc), C.c_int64,
                                                  C.c_int32, vp, P(hh_record)]
            L.hh_gemm_bf16.restype = C.c_int
            L.hh_gemm_bf16.argtypes = [vp, C.c_int32, vp, C.c_int32, vp, C.c_int32, C.c_int32, C.c_int32,
                                       C.c_int32, vp, vp]
            L.hh_surrogate_train.restype = C.c_int
            L.hh_surrogate_train.argtypes = [vp, P(hh_surrogate_desc), P(hh_surrogate_report)]
            L.hh_surrogate_enable.restype = C.c_int
            L.hh_surrogate_enable.argtypes = [vp, C.c_int32]
            L.hh_layer_create.restype = C.c_int
            L.hh_layer_create.argtypes = [P(hh_layer_desc), P(hh_model_desc), P(vp)]
            L.hh_layer_set_weights.restype = C.c_int
            L.hh_layer_set_weights.argtypes = [vp, vp, vp, vp, vp]
            L.hh_layer_forward.restype = C.c_int
            L.hh_layer_forward.argtypes = [vp, vp, vp, vp, vp]
            L.hh_backward.restype = C.c_int
            L.hh_backward.argtypes = [vp, P(hh_grads)]
            L.hh_backward_from.restype = C.c_int
            L.hh_backward_from.argtypes = [vp, C.c_float, vp, vp, vp, P(hh_grads)]
            L.hh_layer_readout.restype = C.c_int
            L.hh_layer_readout.argtypes = [vp, C.c_int32, vp, C.c_size_t, P(C.c_size_t)]
            L.hh_layer_destroy.restype = None
            L.hh_layer_destroy.argtypes = [vp]
            L.hh_destroy.restype = None
            L.hh_destroy.argtypes = [vp]
            L.hh_last_error.restype = C.c_char_p
            L.hh_last_error.argtypes = []
            L.hh_version.restype = C.c_int32
            L.hh_measure_peaks.restype = C.c_int
            L.hh_measure_peaks.argtypes = [P(hh_peaks), vp]
            L.hh_set_wait_limits.restype = C.c_int
            L.hh_set_wait_limits.argtypes = [C.c_int64, C.c_int64]
            L.hh_set_route_pull.restype = C.c_int
            L.hh_set_route_pull.argtypes = [vp, C.c_int64]
            L.hh_poly_fit.restype = C.c_int
            L.hh_poly_fit.argtypes = [P(hh_model_desc), C.c_double, vp, vp, vp, C.c_int64, vp]
            L.hh_state_size.restype = C.c_int
            L.hh_state_size.argtypes = [vp, P(C.c_size_t)]
            L.hh_save_state.restype = C.c_int
            L.hh_save_state.argtypes = [vp, vp, C.c_size_t]
            L.hh_load_state.restype = C.c_int
            L.hh_load_state.argtypes = [vp, vp, C.c_size_t]
            L.hh_set_launch_shape.restype = C.c_int
            L.hh_set_launch_shape.argtypes = [vp, C.c_int32, C.c_int32]
            L.hh_autotune.restype = C.c_int
            L.hh_autotune.argtypes = [vp, C.c_int32, P(hh_tune_report)]
            _lib = L
    return _lib


def _check(status):
    if status != HH_OK:
        raise HHError(status, lib().hh_last_error().decode(errors="replace"))


def hh_last_error() -> str:
    return lib().hh_last_error().decode(errors="replace")


def hh_create_network(desc: hh_net_desc) -> int:
    h = C.c_void_p()
    _check(lib().hh_create_network(C.byref(desc), C.byref(h)))
    return h.value


def hh_set_channels(net: int, model_index: int, model: hh_model_desc, gbar_ptr=None):
    _check(lib().hh_set_channels(net, model_index, C.byref(model), gbar_ptr))


def hh_step_n(net: int, n_steps: int, I_steps_ptr=None, rec: hh_record | None = None):
    _check(lib().hh_step_n(net, n_steps, I_steps_ptr, C.byref(rec) if rec is not None else None))


def hh_reset(net: int, V0_ptr=None):
    _check(lib().hh_reset(net, V0_ptr))


def hh_route_spikes(net: int, step_ptr, idx_ptr, n_spk: int, n_window: int, sumE_ptr, sumI_ptr):
    _check(lib().hh_route_spikes(net, step_ptr, idx_ptr, n_spk, n_window, sumE_ptr, sumI_ptr))


def hh_readout(net: int, what: int, dst_ptr, cap: int) -> int:
    n = C.c_size_t()
    _check(lib().hh_readout(net, what, dst_ptr, cap, C.byref(n)))
    return n.value


def hh_profile(net: int, enable: bool):
    _check(lib().hh_profile(net, 1 if enable else 0))


def hh_step_neurons_noalloc(model: hh_model_desc, state: hh_neurons_noalloc, t0: int, n_steps: int,
                            I_steps_ptr=None, rec: hh_record | None = None):
    _check(lib().hh_step_neurons_noalloc(C.byref(model), C.byref(state), t0, n_steps, I_steps_ptr,
                                         C.byref(rec) if rec is not None else None))


def hh_gemm_bf16(A, Bt, C, M, N, K, splits=1, status=None, stream=None):
    """C[splits][M][N] (fp32) = A[M][K] (bf16) x B (bf16 given as Bt[N][K]);
    torch device tensors."""
    lda = A.stride(0)
    ldb = Bt.stride(0)
    _check(lib().hh_gemm_bf16(A.data_ptr(), lda, Bt.data_ptr(), ldb, C.data_ptr(), M, N, K, splits,
                              status.data_ptr(), stream))


def hh_set_wait_limits(progress_ns: int = -1, mbarrier_polls: int = -1):
    """Bounds of the device-side waits for later launches (-1 = default)."""
    _check(lib().hh_set_wait_limits(int(progress_ns), int(mbarrier_polls)))


def hh_poly_fit(model: dict, dt: float):
    """The HH_PREC_POLY rate tables of a model (host computation): returns
    (interval mV, first V mV, largest relative error, coefficients
    [n_intervals][n_gates][2][4] float32)."""
    info = np.zeros(3, dtype=np.float32)
    n = C.c_int32()
    nf = C.c_int64()
    md = model_desc(model)
    _check(lib().hh_poly_fit(C.byref(md), dt, info.ctypes.data, C.addressof(n), None, 0, C.addressof(nf)))
    c = np.zeros(nf.value, dtype=np.float32)
    _check(lib().hh_poly_fit(C.byref(md), dt, info.ctypes.data, C.addressof(n), c.ctypes.data, c.size,
                             C.addressof(nf)))
    n_gates = sum(len(ch["gates"]) for ch in model["channels"])
    return float(info[0]), float(info[1]), float(info[2]), c.reshape(n.value, n_gates, 2, 4)


def hh_destroy(net: int):
    lib().hh_destroy(net)


def hh_measure_peaks(stream=None) -> dict:
    """FP32 FMA, ex2.approx and rcp.approx results per second on the current
    device (microbenchmarks of the library, CUDA-event timed)."""
    out = hh_peaks()
    _check(lib().hh_measure_peaks(C.byref(out), stream))
    return {"ffma_per_s": out.ffma_per_s, "ex2_per_s": out.ex2_per_s, "rcp_per_s": out.rcp_per_s}


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _fn(t) -> hh_fn:
    form, a, vh, k, vh2, k2, c = t
    return hh_fn(HH_FN[form], a, vh, k, vh2, k2, c)


def model_desc(model: dict) -> hh_model_desc:
    """hh_model_desc from a model table (paper_2601_21407_gb300.inputs)."""
    m = hh_model_desc()
    m.C_m = model["C_m"]
    m.n_channels = len(model["channels"])
    m.ca_channel = -1
    for ci, ch in enumerate(model["channels"]):
        m.channels[ci].E_rev = ch["E"]
        m.channels[ci].gbar = ch["gbar"]
        m.channels[ci].n_gates = len(ch["gates"])
        for gi, g in enumerate(ch["gates"]):
            m.channels[ci].gates[gi] = hh_gate(HH_GATE[g["kind"]], g["power"], _fn(g["f1"]),
                                               _fn(g["f2"]))
    ca = model.get("calcium")
    if ca:
        m.ca_channel = [c["name"] for c in model["channels"]].index(ca["channel"])
        m.ca_tau, m.ca_k, m.ca_rest = ca["tau"], ca["k"], ca["rest"]
    return m


def _ptr(a):
    """Data pointer of a torch tensor or numpy array (None passes through)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class Network:
    """Owns one hh_net.  Arrays may be numpy (host) or torch (host/device);
    the library copies them during creation."""

    def __init__(self, V0, dt, *, I_const=None, model_id=None, csr=None, inh=None, syn=None,
                 delay_steps=1, bg=None, seed=0, theta=0.0, precision=HH_PREC_FAST,
                 v_update=HH_V_EXP_EULER, stream=None, n_nets=1, net_offsets=None,
                 kernels=HH_KERNELS_SPECIALISED, drive=None, morph=None, syn_mode=HH_SYN_CONDUCTANCE):
        d = hh_net_desc()
        self._keep = []
        V0 = self._f32(V0)
        d.n_neurons = int(V0.numel() if hasattr(V0, "numel") else V0.size)
        self.N = d.n_neurons
        d.n_nets = n_nets
        if net_offsets is not None:
            no = np.ascontiguousarray(net_offsets, dtype=np.int64)
            self._keep.append(no)
            d.net_offsets = no.ctypes.data
        d.dt_ms = dt
        d.v_threshold = theta
        d.v_update = v_update
        d.precision = precision
        d.kernels = kernels
        d.V0 = _ptr(V0)
        if I_const is not None:
            I_const = self._f32(I_const)
            d.I_const = _ptr(I_const)
        if model_id is not None:
            model_id = self._arr(model_id, np.uint8)
            d.model_id = _ptr(model_id)
        if csr is not None:
            row_ptr, col, w = csr
            row_ptr = self._arr(row_ptr, np.int64)
            col = self._arr(col, np.int32)
            w = self._f32(w)
            d.n_synapses = int(w.numel() if hasattr(w, "numel") else w.size)
            d.row_ptr, d.col_idx, d.weight = _ptr(row_ptr), _ptr(col), _ptr(w)
        if inh is not None:
            inh = self._arr(inh, np.uint8)
            d.is_inhibitory = _ptr(inh)
        syn = syn or {}
        d.tau_E = syn.get("tau_E", 5.0)
        d.tau_I = syn.get("tau_I", 10.0)
        d.E_E = syn.get("E_E", 0.0)
        d.E_I = syn.get("E_I", -80.0)
        d.area_cm2 = syn.get("area_cm2", 2.0e-4)
        d.delay_steps = delay_steps
        if bg:
            d.bg_rate_hz, d.bg_sources, d.bg_weight_nS = bg["rate_hz"], bg["K"], bg["w"]
            d.bg_weight_sd = bg.get("sd", 0.0)
        d.syn_mode = syn_mode
        d.seed = seed
        d.stream = stream
        if drive is not None:
            # {"amp": [N] uA/cm^2, "freq_hz": [N], "phase": [N] cycles (optional)}
            d.sin_amp = _ptr(self._f32(drive["amp"]))
            d.sin_freq_hz = _ptr(self._f32(drive["freq_hz"]))
            if drive.get("phase") is not None:
                d.sin_phase = _ptr(self._f32(drive["phase"]))
        if morph is not None:
            # {"n_dendrites", "n_per_dendrite", "g_axial", "soma_area_ratio"}
            m = hh_morphology(morph["n_dendrites"], morph["n_per_dendrite"], morph["g_axial"],
                              morph["soma_area_ratio"])
            self._keep.append(m)
            d.morph = C.pointer(m)
        self.handle = hh_create_network(d)
        self._keep = []

    def _arr(self, a, dtype):
        if hasattr(a, "data_ptr"):
            import torch
            tdt = {np.uint8: torch.uint8, np.int32: torch.int32, np.int64: torch.int64,
                   np.float32: torch.float32}[dtype]
            a = a.contiguous().to(tdt)
        else:
            a = np.ascontiguousarray(a, dtype=dtype)
        self._keep.append(a)
        return a

    def _f32(self, a):
        return self._arr(a, np.float32)

    def set_channels(self, model_index, model: dict, gbar=None):
        g = None if gbar is None else self._f32(gbar)
        hh_set_channels(self.handle, model_index, model_desc(model), _ptr(g))
        self._keep = []

    def step(self, n_steps, I_steps=None, rec: hh_record | None = None):
        hh_step_n(self.handle, n_steps, _ptr(I_steps), rec)

    def reset(self, V0=None):
        v = None if V0 is None else self._f32(V0)
        hh_reset(self.handle, _ptr(v))
        self._keep.append(v)

    def state_size(self) -> int:
        n = C.c_size_t(0)
        _check(lib().hh_state_size(self.handle, C.byref(n)))
        return int(n.value)

    def save_state(self, out=None):
        """The full dynamic state (hh_save_state) into `out` (a torch uint8
        tensor on any device, or a numpy uint8 array), or into a new numpy
        array; returns it."""
        n = self.state_size()
        if out is None:
            out = np.zeros(n, dtype=np.uint8)
        nbytes = out.nbytes if hasattr(out, "nbytes") else out.numel() * out.element_size()
        _check(lib().hh_save_state(self.handle, _ptr(out), nbytes))
        return out

    def load_state(self, image):
        nbytes = image.nbytes if hasattr(image, "nbytes") else image.numel() * image.element_size()
        _check(lib().hh_load_state(self.handle, _ptr(image), nbytes))
        self._keep.append(image)

    def set_launch_shape(self, neuron_block=0, route_blocks=0):
        _check(lib().hh_set_launch_shape(self.handle, int(neuron_block), int(route_blocks)))

    def autotune(self, trial_steps=400):
        """hh_autotune: returns {"candidates": [(block, route_blocks, ms)], "best": i}."""
        r = hh_tune_report()
        _check(lib().hh_autotune(self.handle, int(trial_steps), C.byref(r)))
        return {"candidates": [(r.neuron_block[k], r.route_blocks[k], float(r.ms[k])) for k in range(r.n)],
                "best": int(r.best)}

    def route_spikes(self, step, idx, n_window, sumE, sumI):
        hh_route_spikes(self.handle, _ptr(step), _ptr(idx), int(step.numel()), n_window,
                        _ptr(sumE), _ptr(sumI))

    def readout(self, what, dtype=np.float32, count=None):
        sizes = {HH_READ_V: (self.N, np.float32), HH_READ_GATES: (HH_MAX_GATES * self.N, np.float32),
                 HH_READ_CA: (self.N, np.float32), HH_READ_G_SYN: (2 * self.N, np.float32),
                 HH_READ_STATUS: (1, np.int32), HH_READ_TIME: (1, np.int64),
                 HH_READ_N_OUT: (self.N + 1, np.int64), HH_READ_POLY: (3 * HH_MAX_MODELS, np.float32)}
        n, dt = sizes[what]
        out = np.zeros(n, dtype=dt)
        hh_readout(self.handle, what, out.ctypes.data, out.nbytes)
        return out

    def train_surrogate(self, window=10, v_envelope=-55.0, train_neurons=16384, train_windows=1_000_000,
                        epochs=40, batch=8192, lr=2e-3, seed=0, I_min=0.0, I_max=15.0, gbar_sigma=0.3,
                        V0_min=-80.0, V0_max=-55.0, err_V=0.0, err_p=0.0):
        d = hh_surrogate_desc(window, v_envelope, train_neurons, train_windows, epochs, batch, lr, seed,
                              I_min, I_max, gbar_sigma, V0_min, V0_max, err_V, err_p)
        r = hh_surrogate_report()
        _check(lib().hh_surrogate_train(self.handle, C.byref(d), C.byref(r)))
        return {"train_windows": r.train_windows, "train_loss": r.train_loss, "val_loss": r.val_loss,
                "out_scale_V": r.out_scale_V}

    def enable_surrogate(self, enable: bool):
        _check(lib().hh_surrogate_enable(self.handle, 1 if enable else 0))

    def surrogate_stats(self):
        out = np.zeros(2, dtype=np.uint64)
        hh_readout(self.handle, HH_READ_SURROGATE, out.ctypes.data, out.nbytes)
        return int(out[0]), int(out[1])

    def profile(self, enable: bool):
        hh_profile(self.handle, enable)

    def set_route_pull(self, min_spikes: int):
        """Windows with at least min_spikes spikes are routed by a pull over
        the in-CSR (0: every window, < 0: never); hh_set_route_pull."""
        _check(lib().hh_set_route_pull(self.handle, int(min_spikes)))

    def kernel_times(self):
        """{"neuron": (launches, total_ms), "route": (...)} since profile(True)."""
        arr = (hh_kernel_time * HH_KERNEL_COUNT)()
        hh_readout(self.handle, HH_READ_PROFILE, C.addressof(arr), C.sizeof(arr))
        return {"neuron": (arr[0].launches, arr[0].total_ms),
                "route": (arr[1].launches, arr[1].total_ms)}

    def close(self):
        if getattr(self, "handle", None):
            hh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_record(N, n_steps, *, trace=0, trace_idx=None, spike_cap=0, counts=True, device="cuda"):
    """Allocate caller-owned device outputs with torch and an hh_record that
    points at them.  Returns (rec, buffers dict)."""
    import torch
    b = {}
    r = hh_record()
    if trace:
        b["V_trace"] = torch.zeros((n_steps, trace), dtype=torch.float32, device=device)
        r.V_trace = b["V_trace"].data_ptr()
        r.n_trace = trace
        if trace_idx is not None:
            b["trace_idx"] = torch.as_tensor(np.asarray(trace_idx, dtype=np.int32), device=device)
            r.trace_idx = b["trace_idx"].data_ptr()
    if spike_cap:
        b["spikes"] = torch.zeros((spike_cap, 3), dtype=torch.int32, device=device)
        b["n_spikes"] = torch.zeros(1, dtype=torch.int64, device=device)
        r.spikes = b["spikes"].data_ptr()
        r.spike_cap = spike_cap
        r.n_spikes = b["n_spikes"].data_ptr()
    if counts:
        b["counts"] = torch.zeros(N, dtype=torch.int32, device=device)
        r.counts = b["counts"].data_ptr()
    return r, b


def spikes_to_numpy(b):
    """(step, neuron, frac) arrays from a record's spike buffer, sorted by
    (step, neuron)."""
    n = int(b["n_spikes"].item())
    n = min(n, b["spikes"].shape[0])
    raw = b["spikes"][:n].cpu().numpy()
    step = raw[:, 0].copy()
    idx = raw[:, 1].copy()
    frac = raw[:, 2].copy().view(np.float32)
    o = np.lexsort((idx, step))
    return step[o], idx[o], frac[o]


_layer_fn = None


def layer_function():
    """torch.autograd.Function over one Layer: the forward sets the weights
    (hh_layer_set_weights) and runs hh_layer_forward, giving the mean loss
    and the logits; the backward runs hh_backward_from (the hand-derived
    adjoint with recomputation from checkpoints) with the incoming gradient
    of the loss as the weight of the built-in cross-entropy and the incoming
    gradient of the logits as dL/dlogits.  The spike inputs and labels get no
    gradient (layer_spikes_function differentiates X).  The layer's stream
    must be the current torch stream (the default: both are the legacy
    stream), and the backward belongs to the layer's last forward: a later
    forward on the same layer makes an earlier graph's backward raise."""
    global _layer_fn
    if _layer_fn is None:
        import torch

        class _LayerFn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, layer, X, labels, W_in, W_rec, W_out, bias):
                _, B, _, _, n_out = layer.shape
                layer.set_weights(W_in.detach(), W_rec.detach(), W_out.detach(), bias.detach())
                loss = torch.zeros((), dtype=torch.float32, device=X.device)
                logits = torch.zeros((B, n_out), dtype=torch.float32, device=X.device)
                layer.forward(X.contiguous(), labels.to(torch.int32).contiguous(), loss, logits)
                ctx.layer = layer
                ctx.forward_id = layer._forward_id
                ctx.shapes = (tuple(W_in.shape), tuple(W_rec.shape), tuple(W_out.shape), tuple(bias.shape))
                return loss, logits

            @staticmethod
            def backward(ctx, g_loss, g_logits):
                layer = ctx.layer
                if layer._forward_id != ctx.forward_id:
                    raise RuntimeError("the layer ran another forward after this one; its backward is lost")
                dev = (g_loss if g_loss is not None else g_logits).device
                grads = [torch.empty(s, dtype=torch.float32, device=dev) for s in ctx.shapes]
                ce = 0.0 if g_loss is None else float(g_loss.item())
                layer.backward_from(ce_weight=ce, dL_dlogits=None if g_logits is None else g_logits.contiguous(),
                                    dW_in=grads[0], dW_rec=grads[1], dW_out=grads[2], dbias=grads[3])
                return (None, None, None) + tuple(grads)

        _layer_fn = _LayerFn
    return _layer_fn


_spikes_fn = None


def layer_spikes_function():
    """torch.autograd.Function over one Layer whose outputs are the spike
    counts S [T][B][N] and the final membrane potentials V_T [B][N], so that
    any torch loss of them, and any layer in front of X, composes with the
    hand-derived adjoint: the forward sets W_in, W_rec and bias
    (hh_layer_set_weights; the readout weights are zero and unused) and runs
    hh_layer_forward without labels; the backward runs hh_backward_from with
    the incoming gradients as dL/dS and dL/dV and returns dL/dX, dL/dW_in,
    dL/dW_rec and dL/dbias.  X is rounded to bf16 by the input projection
    (exact for 0/1 spikes).  The same stream and last-forward rules as
    layer_function apply."""
    global _spikes_fn
    if _spikes_fn is None:
        import torch

        class _SpikesFn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, layer, X, W_in, W_rec, bias):
                T, B, _, N, n_out = layer.shape
                dev = X.device
                layer.set_weights(W_in.detach(), W_rec.detach(),
                                  torch.zeros((n_out, N), dtype=torch.float32, device=dev), bias.detach())
                layer.forward(X.detach().to(torch.float32).contiguous())
                S = torch.empty((T, B, N), dtype=torch.float32, device=dev)
                V = torch.empty((B, N), dtype=torch.float32, device=dev)
                layer.outputs(S, V)
                ctx.layer = layer
                ctx.forward_id = layer._forward_id
                ctx.shapes = (tuple(X.shape), tuple(W_in.shape), tuple(W_rec.shape), tuple(bias.shape))
                return S, V

            @staticmethod
            def backward(ctx, gS, gV):
                layer = ctx.layer
                if layer._forward_id != ctx.forward_id:
                    raise RuntimeError("the layer ran another forward after this one; its backward is lost")
                dev = gS.device if gS is not None else gV.device
                dX, dW_in, dW_rec, dbias = [torch.empty(s, dtype=torch.float32, device=dev) for s in ctx.shapes]
                layer.backward_from(dL_dS=None if gS is None else gS.contiguous(),
                                    dL_dV=None if gV is None else gV.contiguous(),
                                    dW_in=dW_in, dW_rec=dW_rec, dbias=dbias,
                                    dX=dX if ctx.needs_input_grad[1] else None)
                return (None, dX if ctx.needs_input_grad[1] else None, dW_in, dW_rec, dbias)

        _spikes_fn = _SpikesFn
    return _spikes_fn


class Layer:
    """Owns one hh_layer (differentiable recurrent HH layer).  Device tensors
    are torch tensors; the library does the work."""

    _forward_id = 0

    def __init__(self, model: dict, *, batch, n_in, n_hidden, n_out, n_steps, substeps=10,
                 dt=0.01, theta=0.0, v_init=-65.0, beta=0.5, precision=HH_PREC_FAST, smooth=False,
                 checkpoint_every=25, stream=None):
        d = hh_layer_desc(batch, n_in, n_hidden, n_out, n_steps, substeps, dt, theta, v_init, beta,
                          precision, 1 if smooth else 0, checkpoint_every, stream)
        self.shape = (n_steps, batch, n_in, n_hidden, n_out)
        h = C.c_void_p()
        _check(lib().hh_layer_create(C.byref(d), C.byref(model_desc(model)), C.byref(h)))
        self.handle = h.value

    def set_weights(self, W_in, W_rec, W_out, bias):
        ws = [np.ascontiguousarray(w, dtype=np.float32) if not hasattr(w, "data_ptr") else w.contiguous()
              for w in (W_in, W_rec, W_out, bias)]
        _check(lib().hh_layer_set_weights(self.handle, *[_ptr(w) for w in ws]))

    def forward(self, X, labels=None, loss=None, logits=None):
        _check(lib().hh_layer_forward(self.handle, X.data_ptr(), _ptr(labels), _ptr(loss), _ptr(logits)))
        self._forward_id += 1

    def backward(self, dW_in, dW_rec, dW_out, dbias, dI=None, dX=None):
        g = hh_grads(dW_in.data_ptr(), dW_rec.data_ptr(), dW_out.data_ptr(), dbias.data_ptr(), _ptr(dI),
                     _ptr(dX))
        _check(lib().hh_backward(self.handle, C.byref(g)))

    def backward_from(self, *, ce_weight=0.0, dL_dlogits=None, dL_dS=None, dL_dV=None, dW_in=None,
                      dW_rec=None, dW_out=None, dbias=None, dI=None, dX=None):
        """hh_backward_from: gradients of ce_weight * CE + <dL_dlogits, logits>
        + <dL_dS, S> + <dL_dV, V_T> into the given device tensors."""
        g = hh_grads(_ptr(dW_in), _ptr(dW_rec), _ptr(dW_out), _ptr(dbias), _ptr(dI), _ptr(dX))
        _check(lib().hh_backward_from(self.handle, float(ce_weight), _ptr(dL_dlogits), _ptr(dL_dS),
                                      _ptr(dL_dV), C.byref(g)))

    def outputs(self, spikes, V):
        """Copy the last forward's spikes [T][B][N] and final V [B][N] into
        the given fp32 tensors (device or host; synchronous)."""
        n = C.c_size_t()
        _check(lib().hh_layer_readout(self.handle, HH_LAYER_SPIKES, spikes.data_ptr(),
                                      spikes.numel() * 4, C.byref(n)))
        _check(lib().hh_layer_readout(self.handle, HH_LAYER_V, V.data_ptr(), V.numel() * 4, C.byref(n)))

    def spikes(self, X, W_in, W_rec, bias):
        """The layer as a differentiable torch function of its inputs and
        weights (see layer_spikes_function): returns (S [T][B][N], V_T [B][N])."""
        return layer_spikes_function().apply(self, X, W_in, W_rec, bias)

    def loss(self, X, labels, W_in, W_rec, W_out, bias):
        """The mean cross-entropy loss as a differentiable torch function of
        the weights (see layer_function); returns (loss, logits)."""
        return layer_function().apply(self, X, labels, W_in, W_rec, W_out, bias)

    def readout(self, what):
        T, B, _, N, _ = self.shape
        n = {HH_LAYER_SPIKES: T * B * N, HH_LAYER_V: B * N, HH_LAYER_STATUS: 1}[what]
        out = np.zeros(n, dtype=np.int32 if what == HH_LAYER_STATUS else np.float32)
        nb = C.c_size_t()
        _check(lib().hh_layer_readout(self.handle, what, out.ctypes.data, out.nbytes, C.byref(nb)))
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().hh_layer_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
