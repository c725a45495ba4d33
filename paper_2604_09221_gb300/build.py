"""Build libtcurve.so in-tree with nvcc for sm_103a (GB300).

The library is the C ABI of include/tcurve.h: host.cpp (validation, tables,
object management) and kernels.cu (the sm_103a kernels), linked against the
shared CUDA runtime so that it shares the runtime instance of the host
process (e.g. PyTorch's) and accepts its streams.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libtcurve.so")
SOURCES = ["host.cpp", "kernels.cu", "warp_kernels.cu", "jit.cpp", "noalloc.cu", "batch.cu", "fused.cu",
           "int_peak.cu"]
HEADERS = ["engine.h", "tc_layout.h", "tc_runtime.cuh", "tc_table_sweep.cuh", "tc_warp_sweep.cuh",
           "tc_stage.cuh", "jit_kernels.cuh",
           os.path.join("..", "..", "include", "tcurve.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [__file__]
    return any(os.path.getmtime(p) > t for p in deps)


def embed_device_runtime() -> None:
    """Write the device runtime (tc_runtime.cuh) and the kernels of the
    specialised sources (jit_kernels.cuh) as C++ raw string literals, which
    jit.cpp puts around the code it generates for a triangulation."""
    for name in ("tc_runtime", "jit_kernels"):
        src = open(os.path.join(CSRC, name + ".cuh")).read()
        out = os.path.join(OUT_DIR, f"_{name}_src.inc")
        text = 'R"TCJIT(' + src + ')TCJIT"\n'
        if not os.path.exists(out) or open(out).read() != text:
            with open(out, "w") as f:
                f.write(text)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the sources (in parallel) and link libtcurve.so; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    embed_device_runtime()
    tmp = tempfile.mkdtemp(prefix="tcurve_build_", dir=OUT_DIR)
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              *ARCH, f"-I{CSRC}", f"-I{OUT_DIR}"]
    procs, objs = [], []
    try:
        for s in SOURCES:
            obj = os.path.join(tmp, s + ".o")
            cmd = [nvcc(), *common, "-c", os.path.join(CSRC, s), "-o", obj]
            if s.endswith(".cu"):
                cmd += ["-Xptxas", "-v"] if verbose else []
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
            objs.append(obj)
        for cmd, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + out.decode(errors="replace"))
            if verbose and out:
                print(out.decode(errors="replace"))
        out_tmp = os.path.join(tmp, "libtcurve.so")
        subprocess.check_call([nvcc(), "-shared", *ARCH, "-cudart", "shared", "-o", out_tmp, *objs,
                               "-ldl"])
        os.replace(out_tmp, LIB)
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
