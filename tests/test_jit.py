"""CPU tests of the runtime-compiled pass kernels (no GPU).

tests/jit_check.cpp is compiled with the host compiler against the
library's planner, op validation and kernel generator, and NVRTC.  For each
gate list it plans the passes, generates the kernel source of every pass
(the generator refuses forms it does not know) and compiles a capped number
of the distinct kernels for sm_103a, so every operation family the planner
emits is shown to compile without a GPU.  What the kernels compute is
checked on the GPU (tests/test_gpu_jit.py: bit-identical to the
interpreting kernel, and against the oracle).
"""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_1802_08032_b300 import circuits as C
from paper_1802_08032_b300 import qsim as Q
from paper_1802_08032_b300 import build as B

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1802_08032_b300", "csrc")
CUDA = "/usr/local/cuda"


@pytest.fixture(scope="session")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA, "include", "nvrtc.h")):
        pytest.skip("host compiler or NVRTC missing")
    gen = str(tmp_path_factory.mktemp("jitgen"))
    B.write_jit_headers(gen)
    exe = os.path.join(gen, "jit_check")
    srcs = [os.path.join(HERE, "jit_check.cpp")] + [os.path.join(CSRC, f) for f in
                                                    ("planner.cpp", "oplist.cpp", "jit_gen.cpp", "jit.cpp")]
    subprocess.check_call([cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                           "-I", gen, "-I", os.path.join(CUDA, "include"), "-o", exe, *srcs,
                           "-L", os.path.join(CUDA, "lib64"), "-lnvrtc", "-lcudart", "-lpthread"])
    return exe


def run(exe, n, ops, density=False, prec=128, arith=0, k_req=0, ctas=2, max_compile=4, copy=0, tile_low=0):
    arr, cnt = Q.to_qsops(ops)
    data = ctypes.string_at(ctypes.addressof(arr), ctypes.sizeof(Q.QSOp) * cnt)
    env = dict(os.environ)
    env["JIT_CHECK_TILE_LOW"] = str(tile_low)
    env["LD_LIBRARY_PATH"] = os.path.join(CUDA, "lib64") + ":" + env.get("LD_LIBRARY_PATH", "")
    r = subprocess.run([exe, str(n), str(int(density)), str(prec), str(arith), str(k_req), str(ctas),
                        str(copy), str(max_compile)], input=data, capture_output=True, timeout=600, env=env)
    out = r.stdout.decode(errors="replace")
    assert r.returncode == 0, out[-3000:] + r.stderr.decode(errors="replace")[-2000:]
    head = out.strip().splitlines()[-1]
    assert head.startswith("JIT passes"), out
    f = head.split()
    return int(f[2]), int(f[4]), int(f[6])


def extras(n, seed):
    rng = C.SplitMix64(seed)
    ops = []
    for _ in range(2 * n):
        qs = C.distinct_qubits(rng, n, 3)
        a = C.haar_alpha_beta(rng)
        al, be = complex(a[0], a[1]), complex(a[2], a[3])
        u = (al.real, al.imag, -be.real, be.imag, be.real, be.imag, al.real, -al.imag)
        k = rng.below(5)
        ops.append([C.Op("CNOT", (qs[0],), (qs[1],)), C.Op("CUNITARY", (qs[0],), tuple(qs[1:]), u),
                    C.Op("PHASE", (qs[0],), (), (0.3 + rng.uniform(),)), C.Op("X", (qs[0],)),
                    C.Op("UNITARY", (qs[0],), (), u)][k])
    return ops


@pytest.mark.parametrize("prec,arith", [(64, 0), (128, 0), (128, 1)])
def test_30_qubit_workload_passes_generate_and_compile(harness, prec, arith):
    passes, compiled, distinct = run(harness, 30, C.workload_30q(), prec=prec, arith=arith,
                                     max_compile=3 if arith == 0 else 2)
    assert passes > 0 and distinct == passes and compiled >= 2


@pytest.mark.parametrize("prec,arith", [(64, 0), (128, 0), (128, 1)])
def test_controlled_gates_and_small_tiles(harness, prec, arith):
    n = 15
    ops = C.random_circuit(n, 12, 77, extras=True) + extras(n, 9)
    for k in (0, 9):
        passes, compiled, _ = run(harness, n, ops[len(ops) // 4:], prec=prec, arith=arith, k_req=k,
                                  max_compile=2)
        assert passes > 0 and compiled >= 1


@pytest.mark.parametrize("arith", [0, 1])
def test_density_matrix_passes(harness, arith):
    N = 7
    ops = C.with_noise(C.random_circuit(N, 10, 31, extras=True) + extras(N, 3), 0.3, 0.6)
    passes, compiled, _ = run(harness, N, ops, density=True, arith=arith, max_compile=3)
    assert passes > 0 and compiled >= 1


def test_three_ctas_per_sm_compiles(harness):
    passes, compiled, _ = run(harness, 24, C.workload_30q(24), prec=64, ctas=3, max_compile=2)
    assert compiled == 2


@pytest.mark.parametrize("copy", [1, 2, 4, 6, 8, 14])
@pytest.mark.parametrize("prec,arith,k", [(64, 0, 12), (64, 0, 13), (128, 0, 11), (128, 1, 11)])
def test_copy_pipelines_compile(harness, prec, arith, k, copy):
    """The bulk-copy (TMA) and async-copy double-buffered forms, (copy + 4)
    the last stage storing straight to HBM, (copy + 8) without the
    shared-memory swizzle."""
    passes, compiled, _ = run(harness, 26, C.workload_30q(26), prec=prec, arith=arith, k_req=k, copy=copy,
                              max_compile=2)
    assert compiled == 2


@pytest.mark.parametrize("copy", [1, 2])
def test_copy_pipelines_density_small_tiles(harness, copy):
    N = 7
    ops = C.with_noise(C.random_circuit(N, 10, 31, extras=True) + extras(N, 3), 0.3, 0.6)
    passes, compiled, _ = run(harness, N, ops, density=True, k_req=9, copy=copy, max_compile=2)
    assert compiled >= 1


@pytest.mark.parametrize("tile_low", [2, 3])
@pytest.mark.parametrize("prec,arith,copy", [(64, 0, 2), (64, 0, 6), (64, 0, 1), (128, 0, 0), (128, 1, 4)])
def test_passes_with_fewer_low_tile_qubits_compile(harness, tile_low, prec, arith, copy):
    """Plans whose tiles hold 2 or 3 contiguous low qubits ("tile_low_qubits":
    HBM chunks of 32 / 64 bytes for complex64) generate kernels that compile
    in every copy form, the bulk copies included (chunks stay a multiple of
    16 bytes)."""
    passes, compiled, _ = run(harness, 26, C.workload_30q(26), prec=prec, arith=arith,
                              k_req=12 if prec == 64 else 0, copy=copy, max_compile=2, tile_low=tile_low)
    assert passes > 0 and compiled == 2
