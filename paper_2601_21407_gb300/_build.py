"""Build libhh.so in-tree with nvcc for sm_103a (no torch extension, no cmake).

The translation units are compiled in parallel, then linked into a shared
library next to this file.  Host code is compiled without floating-point
contraction so that host-side tables (the Poisson thresholds) are computed
with the same operation sequence on x86 and Arm hosts.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhh.so")
# (source, object, extra flags): the table-interpreting kernels are compiled
# once per precision so that their instantiations build in parallel
UNITS = [(f, f.replace(".cu", ".o"), []) for f in
         ("hh_kernels.cu", "hh_abi.cu", "hh_jit.cu", "hh_gemm.cu", "hh_layer.cu", "hh_surrogate.cu", "hh_peaks.cu")]
UNITS += [("hh_table.cu", f"hh_table_{p}.o", [f"-DHH_TABLE_PREC={p}"]) for p in (0, 1, 2)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "hh.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    # the shared device code is compiled into the library and also embedded
    # verbatim for the run-time (NVRTC) specialisation of the neuron and
    # layer kernels
    for name in ("hh_device", "hh_layer_device"):
        src = open(os.path.join(CSRC, name + ".cuh")).read()
        assert ')HHSRC"' not in src
        with open(os.path.join(BUILD, name + "_src.inc"), "w") as f:
            f.write('R"HHSRC(' + src + ')HHSRC"\n')
    cc = nvcc()
    cuda_home = os.path.dirname(os.path.dirname(os.path.realpath(cc)))
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-I", os.path.join(HERE, "..", "include"), "-I", BUILD]
    if ptxas_info:
        common += ["-Xptxas", "-v"]
    procs, objs = [], []
    for src, obj_name, flags in UNITS:
        obj = os.path.join(BUILD, obj_name)
        objs.append(obj)
        cmd = [cc, "-c", os.path.join(CSRC, src), "-o", obj] + common + flags
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    logs = []
    for cmd, p in procs:
        out, _ = p.communicate()
        logs.append(out.decode(errors="replace"))
        if p.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + logs[-1])
    tmp = LIB + f".{os.getpid()}.tmp"
    libdir = os.path.join(cuda_home, "lib64")
    link = [cc, "-shared"] + ARCH + objs + ["-o", tmp, "-lcudart", "-lnvrtc", "-L", libdir,
                                            "-Xlinker", f"-rpath,{libdir}"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    if verbose or ptxas_info:
        for l in logs:
            if l.strip():
                print(l, file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
