"""The C-ABI library builds, loads, exports every declared symbol, its structs
match the ctypes mirrors, and host-side argument checks fire (CPU only: no
compute call needs a GPU here)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2601_21407_gb300 import hh, inputs as inp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hh.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hh_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    L = hh.lib()
    names = declared_functions()
    assert set(names) == set(hh.EXPORTS)
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", hh.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}$", out, re.M), n


def test_struct_layout_matches_header(tmp_path):
    """Compile a probe against include/hh.h with gcc and compare sizes and
    offsets with the ctypes mirrors."""
    probe = tmp_path / "probe.c"
    probe.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "hh.h"
int main(void){
 printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(hh_fn), sizeof(hh_gate), sizeof(hh_channel),
   sizeof(hh_model_desc), sizeof(hh_net_desc), sizeof(hh_record), sizeof(hh_spike));
 printf("%zu %zu\\n", sizeof(hh_neurons_noalloc), offsetof(hh_neurons_noalloc, status));
 printf("%zu %zu %zu %zu %zu\\n", offsetof(hh_net_desc, dt_ms), offsetof(hh_net_desc, n_synapses),
   offsetof(hh_net_desc, seed), offsetof(hh_net_desc, stream), offsetof(hh_model_desc, ca_tau));
 printf("%zu %zu %zu %zu\\n", offsetof(hh_net_desc, V0), offsetof(hh_net_desc, sin_phase),
   offsetof(hh_net_desc, morph), sizeof(hh_morphology));
 printf("%zu %zu\\n", offsetof(hh_net_desc, bg_weight_sd), sizeof(hh_net_desc));
 printf("%zu %zu\\n", sizeof(hh_peaks), offsetof(hh_peaks, rcp_per_s));
 printf("%zu %zu\\n", sizeof(hh_grads), offsetof(hh_grads, dX));
 printf("%zu %zu\\n", sizeof(hh_tune_report), offsetof(hh_tune_report, ms));
 printf("%zu %zu\\n", sizeof(hh_surrogate_desc), offsetof(hh_surrogate_desc, err_p));
 return 0; }
""")
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(probe), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    want = [C.sizeof(hh.hh_fn), C.sizeof(hh.hh_gate), C.sizeof(hh.hh_channel),
            C.sizeof(hh.hh_model_desc), C.sizeof(hh.hh_net_desc), C.sizeof(hh.hh_record),
            C.sizeof(hh.hh_spike), C.sizeof(hh.hh_neurons_noalloc),
            hh.hh_neurons_noalloc.status.offset, hh.hh_net_desc.dt_ms.offset, hh.hh_net_desc.n_synapses.offset,
            hh.hh_net_desc.seed.offset, hh.hh_net_desc.stream.offset,
            hh.hh_model_desc.ca_tau.offset, hh.hh_net_desc.V0.offset, hh.hh_net_desc.sin_phase.offset,
            hh.hh_net_desc.morph.offset, C.sizeof(hh.hh_morphology),
            hh.hh_net_desc.bg_weight_sd.offset, C.sizeof(hh.hh_net_desc),
            C.sizeof(hh.hh_peaks), hh.hh_peaks.rcp_per_s.offset,
            C.sizeof(hh.hh_grads), hh.hh_grads.dX.offset,
            C.sizeof(hh.hh_tune_report), hh.hh_tune_report.ms.offset,
            C.sizeof(hh.hh_surrogate_desc), hh.hh_surrogate_desc.err_p.offset]
    assert got == want


def _desc(**kw):
    d = hh.hh_net_desc()
    V0 = np.full(4, -65.0, dtype=np.float32)
    d.n_neurons = 4
    d.n_nets = 1
    d.dt_ms = 0.01
    d.V0 = V0.ctypes.data
    for k, v in kw.items():
        setattr(d, k, v)
    return d, V0


@pytest.mark.parametrize("field,value", [("n_neurons", 0), ("dt_ms", 0.0), ("dt_ms", -1.0),
                                         ("n_nets", 0), ("precision", 7), ("v_update", 3),
                                         ("kernels", 3), ("kernels", -1), ("V0", None)])
def test_create_rejects_bad_descriptor(field, value):
    d, keep = _desc(**{field: value})
    h = C.c_void_p()
    st = hh.lib().hh_create_network(C.byref(d), C.byref(h))
    assert st == hh.HH_EINVAL
    assert h.value is None
    assert hh.hh_last_error()


def test_null_arguments():
    L = hh.lib()
    assert L.hh_create_network(None, None) == hh.HH_EINVAL
    assert L.hh_step_n(None, 1, None, None) == hh.HH_EINVAL
    assert L.hh_reset(None, None) == hh.HH_EINVAL
    assert L.hh_readout(None, 0, None, 0, None) == hh.HH_EINVAL
    assert L.hh_set_channels(None, 0, None, None) == hh.HH_EINVAL
    L.hh_destroy(None)


def test_null_arguments_of_state_and_launch_shape_calls():
    """Checkpoint, launch-shape and autotuning calls reject a NULL network or
    buffer before touching the device."""
    L = hh.lib()
    n = C.c_size_t(0)
    buf = (C.c_uint8 * 512)()
    assert L.hh_state_size(None, C.byref(n)) == hh.HH_EINVAL
    assert L.hh_save_state(None, buf, 512) == hh.HH_EINVAL
    assert L.hh_load_state(None, buf, 512) == hh.HH_EINVAL
    assert L.hh_set_launch_shape(None, 0, 0) == hh.HH_EINVAL
    assert L.hh_autotune(None, 100, None) == hh.HH_EINVAL
    rep = hh.hh_surrogate_report()
    assert L.hh_surrogate_train(None, None, C.byref(rep)) == hh.HH_EINVAL
    assert hh.hh_last_error()


def test_model_marshalling_roundtrip():
    m = hh.model_desc(inp.MULTI_CHANNEL)
    assert m.n_channels == len(inp.MULTI_CHANNEL["channels"])
    assert m.ca_channel == 3
    assert m.channels[0].gates[0].f1.form == hh.HH_FN["linoid"]
    assert m.channels[2].gates[1].f2.form == hh.HH_FN["bell"]
    assert m.channels[0].gates[0].power == 3


def test_measure_peaks_rejects_null():
    assert hh.lib().hh_measure_peaks(None, None) == hh.HH_EINVAL
    assert "NULL" in hh.hh_last_error()
