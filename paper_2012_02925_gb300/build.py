"""Build the CUDA library (libfvgb.so) in-tree for sm_103a with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfvgb.so")
# the stage kernel variants (fv_stage_<form>[_fast][_visc][_bc].cu, one per
# translation unit so that they compile in parallel), then the rest
STAGE_VARIANTS = [form + fast + visc + bc for form in ("fp64", "df64", "fp32") for fast in ("", "_fast")
                  for visc in ("", "_visc") for bc in ("", "_bc")]
SOURCES = ["fv_stage_%s.cu" % v for v in STAGE_VARIANTS] + [
    "fv_api.cu", "fv_noalloc.cu", "fv_probe.cu", "fv_adjoint.cu", "fv_visc.cu", "fv_monitor.cu"]
HEADERS = ["fv_arith.cuh", "fv_face.cuh", "fv_stage.cuh", "fv_viscface.cuh", "fv_internal.h", "fv_adjoint.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cuda, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "fvgb.h")]
    nvcc = _nvcc()

    def compile_one(src):
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc] + ARCH + FLAGS + ["-c", s, "-o", o + ".tmp"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr))
            with open(os.path.join(BUILD, src + ".ptxas.txt"), "w") as f:
                f.write(r.stderr)
            os.replace(o + ".tmp", o)
        return o

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), max(4, os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if force or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
