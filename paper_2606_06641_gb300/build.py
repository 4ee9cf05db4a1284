"""Builds the in-tree shared library libafsat.so for sm_103a.

Every translation unit under csrc/ is compiled in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a``), then linked into
``_lib/libafsat.so`` with the CUDA runtime linked statically. The short
FE+gradient kernel's dispatch (csrc/short_dispatch.cuh) is instantiated in
four generated translation units, one per (basis, state type), written to
``_build/gen/`` so that they compile in parallel. Objects live in ``_build/``;
a unit is recompiled when it or any header is newer than its object.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libafsat.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-O2", f"-I{INCLUDE}", f"-I{CSRC}"]
SOURCES = ["host.cpp", "coef.cpp", "kernels.cu", "long_pgf.cu", "persist.cu", "noalloc.cu", "mpnn.cu"]
# generated units: (name, state type, paper basis)
SHORT_UNITS = [("short_pgf_f32", "float", "false"), ("short_pgf_bf16", "__nv_bfloat16", "false"),
               ("short_esp_f32", "float", "true"), ("short_esp_bf16", "__nv_bfloat16", "true")]


def _generate_short_units() -> list:
    gen = os.path.join(BUILD_DIR, "gen")
    os.makedirs(gen, exist_ok=True)
    paths = []
    for name, xt, esp in SHORT_UNITS:
        text = ("// generated by build.py: the short kernel's dispatch for one (basis, state type)\n"
                '#include "short_dispatch.cuh"\n'
                f"namespace afs {{\nbool launch_{name}(const FeGroupArgs& a, int rpl, int warps, cudaStream_t s) {{\n"
                f"  return launch_short<{xt}, {esp}>(a, rpl, warps, s);\n}}\n}}  // namespace afs\n")
        p = os.path.join(gen, name + ".cu")
        old = open(p).read() if os.path.exists(p) else None
        if old != text:
            with open(p, "w") as fh:
                fh.write(text)
        paths.append(p)
    return paths


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libafsat")


def _headers_mtime() -> float:
    hs = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(h) for h in hs)


def build(verbose: bool = False, force: bool = False, jobs: int = 0) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    hdr = _headers_mtime()
    todo = []
    objs = []
    for sp in [os.path.join(CSRC, src) for src in SOURCES] + _generate_short_units():
        op = os.path.join(BUILD_DIR, os.path.basename(sp) + ".o")
        objs.append(op)
        if force or not os.path.exists(op) or os.path.getmtime(op) < max(os.path.getmtime(sp), hdr):
            todo.append((sp, op))

    def compile_one(item):
        sp, op = item
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", sp, "-o", op]
        if sp.endswith(".cpp"):
            cmd.insert(1, "-x")
            cmd.insert(2, "c++")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return op

    if todo:
        with ThreadPoolExecutor(max_workers=jobs or min(len(todo), os.cpu_count() or 4)) as ex:
            list(ex.map(compile_one, todo))
    if todo or not os.path.exists(LIB_PATH):
        tmp = LIB_PATH + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    import sys
    print(build(verbose=True, force="--force" in sys.argv))
