"""Build the in-tree CUDA library libracecheck.so for sm_103a.

Every translation unit is compiled in parallel with nvcc (one -gencode,
sm_103a only) and linked into paper_1308_3203_gb300/libracecheck.so.  Objects
go to paper_1308_3203_gb300/_build/.  No cmake, no torch extension machinery.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libracecheck.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}", f"-I{OUT_DIR}"]
SOURCES = ["compiler.cpp", "features.cpp", "prove.cpp", "interp.cu", "sort.cu", "classify.cu", "shadow.cu", "runtime.cu",
           "noalloc.cu", "batch.cu", "mlp.cu", "explore.cu", "xgroup.cu", "translate.cpp", "jit.cu"]
# headers compiled at run time into the kernels of compiled intervals (NVRTC):
# embedded into the library as string literals
JIT_HEADERS = ["isa.h", "kernel_types.cuh", "semantics.cuh", "interp_kernel.cuh", "jit_engine.cuh"]


def _nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libracecheck.so")
    return p


def _deps():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    out += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return out + [os.path.abspath(__file__)]


def up_to_date() -> bool:
    return os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(d) for d in _deps())


def write_jit_headers() -> None:
    """_build/jit_headers.inc: the engine headers as C string literals."""
    names, texts = [], []
    for h in JIT_HEADERS:
        text = open(os.path.join(CSRC, h), encoding="utf-8").read()
        assert ")RCJIT\"" not in text
        names.append(f'"{h}"')
        texts.append('R"RCJIT(' + text + ')RCJIT"')
    out = (f"constexpr unsigned kJitHeaderCount = {len(names)};\n"
           f"const char *const kJitHeaderNames[] = {{{', '.join(names)}}};\n"
           "const char *const kJitHeaderTexts[] = {\n" + ",\n".join(texts) + "};\n")
    path = os.path.join(OUT_DIR, "jit_headers.inc")
    if not os.path.exists(path) or open(path, encoding="utf-8").read() != out:
        with open(path, "w", encoding="utf-8") as f:
            f.write(out)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    write_jit_headers()
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        objs.append(obj)
        cmd = [nvcc] + NVFLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "c++"] + NVFLAGS[len(ARCH):] + ["-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed on {failed}")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-ldl"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
