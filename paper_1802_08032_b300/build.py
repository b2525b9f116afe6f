"""Builds the CUDA library libqsim.so in-tree for sm_103a with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libqsim.so")
SOURCES = ["api.cu", "oplist.cpp", "launch.cu", "planner.cpp", "fused.cu", "profiler.cu", "noalloc.cu",
           "batch.cu", "serve.cu", "jit.cpp", "jit_gen.cpp", "partition.cpp", "partition.cu"]
# device headers the runtime-compiled pass kernels include (embedded in the
# library for NVRTC)
JIT_HEADERS = ["common.cuh", "dfloat.cuh", "fused_types.h", "pair_arith.cuh", "fused_arith.cuh", "mbarrier.cuh"]
GEN = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(ROOT, "include", "qsim.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def write_jit_headers(out_dir: str = GEN) -> str:
    """Writes jit_headers.inc: the JIT_HEADERS sources as C++ raw string
    literals, {name, text} pairs in an array kJitHeaders."""
    os.makedirs(out_dir, exist_ok=True)
    parts = []
    for name in JIT_HEADERS:
        with open(os.path.join(CSRC, name)) as f:
            text = f.read()
        assert ")QSJIT\"" not in text
        parts.append(f'  {{"{name}", R"QSJIT({text})QSJIT"}},')
    body = "const EmbeddedHeader kJitHeaders[] = {\n" + "\n".join(parts) + "\n};\n"
    path = os.path.join(out_dir, "jit_headers.inc")
    old = open(path).read() if os.path.exists(path) else None
    if old != body:
        with open(path + ".tmp", "w") as f:
            f.write(body)
        os.replace(path + ".tmp", path)
    return path


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    """Compiles every source to an object (in parallel), then links
    libqsim.so; each translation unit is self-contained (no device code is
    linked across units)."""
    if not force and not _stale():
        return LIB
    write_jit_headers()
    common = [nvcc(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC",
              "-I", os.path.join(ROOT, "include"), "-I", GEN, *extra]
    tag = f"{os.getpid()}"
    objs = [os.path.join(GEN, f"{s.replace('.', '_')}.{tag}.o") for s in SOURCES]
    cmds = [common + ["-c", "-o", o, os.path.join(CSRC, s)] for s, o in zip(SOURCES, objs)]
    if verbose:
        for c in cmds:
            print(" ".join(c), file=sys.stderr)
    from concurrent.futures import ThreadPoolExecutor
    tmp = LIB + f".tmp{tag}"
    try:
        with ThreadPoolExecutor(max_workers=max(1, min(len(cmds), os.cpu_count() or 1))) as ex:
            for f in [ex.submit(subprocess.check_call, c) for c in cmds]:
                f.result()
        link = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-lnvrtc"]
        if verbose:
            print(" ".join(link), file=sys.stderr)
        subprocess.check_call(link)
        os.replace(tmp, LIB)
    finally:
        for o in objs + [tmp]:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else []))
