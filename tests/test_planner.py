"""CPU tests of the fused-pass planner (host logic, no GPU).

tests/planner_check.cpp is compiled with the host compiler against the
library's planner and op-validation sources.  For each gate list it plans
the passes, checks the invariants the fused kernel relies on (tile qubits,
R distinct ascending register positions per stage, condition masks that
split cleanly into register / local / global bits, dispatch codes) and
applies the encoded passes to |0...0> on the CPU.  The result must match
the oracle: this pins the planner and the operation encoding (unscaled
H / sqrt(X) / sqrt(Y) with the deferred scale factor, pending sign flips,
per-thread and per-tile conditions, the density-matrix column updates of
Eq. 2) independently of the GPU.
"""
import os
import shutil
import subprocess
import ctypes

import numpy as np
import pytest

from paper_1802_08032_b300 import circuits as C
from paper_1802_08032_b300 import qsim as Q
from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1802_08032_b300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


@pytest.fixture(scope="session")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("host compiler or CUDA headers missing")
    exe = str(tmp_path_factory.mktemp("planner") / "planner_check")
    srcs = [os.path.join(HERE, "planner_check.cpp"), os.path.join(CSRC, "planner.cpp"),
            os.path.join(CSRC, "oplist.cpp")]
    base = [cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", CUDA_INC,
            "-o", exe, *srcs]
    # undefined behaviour in the planner (shifts, overflows) aborts the run
    ubsan = ["-fsanitize=undefined", "-fno-sanitize-recover=undefined"]
    if subprocess.run(base[:1] + ubsan + base[1:], capture_output=True).returncode != 0:
        subprocess.check_call(base)
    return exe


def run(exe, n, ops, density=False, prec=128, arith=0, k_req=0, emulate=True, tile_low=0):
    arr, cnt = Q.to_qsops(ops)
    data = ctypes.string_at(ctypes.addressof(arr), ctypes.sizeof(QSOp) * cnt)
    r = subprocess.run([exe, str(n), str(int(density)), str(prec), str(arith), str(k_req),
                        str(int(emulate)), "1", str(tile_low)], input=data, capture_output=True, timeout=120)
    out = r.stdout
    head, _, rest = out.partition(b"\n")
    assert r.returncode == 0, (head.decode(), r.stderr.decode()[-2000:])
    assert b"violations 0" in head, head
    if not emulate:
        return head.decode(), None
    tag, _, body = rest.partition(b"\n")
    assert tag == b"STATE"
    return head.decode(), np.frombuffer(body, dtype=np.complex128)


QSOp = Q.QSOp
TOL = {(128, 0): 1e-12, (128, 1): 1e-12, (64, 0): 1e-5}


def controlled_extras(n, seed):
    """CNOT, controlled and multi-controlled unitaries, phase shifts (the
    random layering has none of them)."""
    rng = C.SplitMix64(seed)
    ops = []
    for _ in range(3 * n):
        qs = C.distinct_qubits(rng, n, min(n, 3))
        a = C.haar_alpha_beta(rng)
        al, be = complex(a[0], a[1]), complex(a[2], a[3])
        u = (al.real, al.imag, -be.real, be.imag, be.real, be.imag, al.real, -al.imag)
        kind = rng.below(4)
        if kind == 0 and n >= 2:
            ops.append(C.Op("CNOT", (qs[0],), (qs[1],)))
        elif kind == 1 and n >= 2:
            ops.append(C.Op("CUNITARY", (qs[0],), tuple(qs[1:]), u))
        elif kind == 2:
            ops.append(C.Op("PHASE", (qs[0],), (), (0.3 + rng.uniform(),)))
        else:
            ops.append(C.Op("UNITARY", (qs[0],), (), u))
    return ops


@pytest.mark.parametrize("n", [1, 3, 5, 8, 11, 13, 14])
@pytest.mark.parametrize("prec,arith", [(128, 0), (128, 1), (64, 0)])
def test_planned_state_vector_matches_oracle(harness, n, prec, arith):
    ops = C.random_circuit(n, 10, 100 + n, extras=n >= 3)
    ops = ops[: len(ops) // 2] + controlled_extras(n, n) + ops[len(ops) // 2:]
    if n < (5 if prec == 64 else 4):
        pytest.skip("registers below R qubits (5 complex64, 4 complex128) are not fused")
    head, psi = run(harness, n, ops, prec=prec, arith=arith)
    ref = O.run_circuit(n, ops).a
    assert np.max(np.abs(psi - ref)) <= TOL[(prec, arith)], head


@pytest.mark.parametrize("n,k", [(14, 9), (13, 9), (12, 10), (14, 11)])
@pytest.mark.parametrize("part", ["whole", "suffix"])
def test_tile_smaller_than_register(harness, n, k, part):
    """Qubits outside the tile: per-tile conditions, phases and flips whose
    qubits are global, and stage register sets that must still be R tile
    positions.  A suffix of a circuit (as a later flush of the same register
    sees it) has phases before any other op on their qubits, so they land in
    passes whose tile does not hold them."""
    ops = C.random_circuit(n, 12, 7 * n + k, extras=True) + controlled_extras(n, k)
    if part == "suffix":
        ops = ops[len(ops) // 3:]
    head, psi = run(harness, n, ops, k_req=k)
    assert f" k {k} " in head, head
    ref = O.run_circuit(n, ops).a
    assert np.max(np.abs(psi - ref)) <= 1e-12, head


@pytest.mark.parametrize("N", [2, 4, 6])
@pytest.mark.parametrize("arith", [0, 1])
def test_planned_density_matrix_matches_oracle(harness, N, arith):
    ops = C.random_density_circuit(N, 8, 40 + N, 0.01, 0.005)
    head, rho = run(harness, N, ops, density=True, arith=arith, k_req=0)
    ref = O.run_circuit(N, ops, density=True).a
    assert np.max(np.abs(rho - ref)) <= 1e-12, head


@pytest.mark.parametrize("N", [3, 5])
@pytest.mark.parametrize("arith", [0, 1])
def test_planned_density_matrix_general_gates(harness, N, arith):
    """General, controlled and phase gates on a density matrix: the column
    updates carry conjugated matrices through absorption, the phase-shear-
    phase form and the unscaled phases."""
    gates = C.random_circuit(N, 6, 90 + N, extras=True) + controlled_extras(N, N + 1)
    ops = C.with_noise(gates, 0.02, 0.01)
    head, rho = run(harness, N, ops, density=True, arith=arith)
    ref = O.run_circuit(N, ops, density=True).a
    assert np.max(np.abs(rho - ref)) <= 1e-12, head


def test_density_matrix_small_tile(harness):
    N = 6
    ops = C.random_density_circuit(N, 6, 77, 0.02, 0.01)
    head, rho = run(harness, N, ops, density=True, k_req=9)
    ref = O.run_circuit(N, ops, density=True).a
    assert np.max(np.abs(rho - ref)) <= 1e-12, head


@pytest.mark.parametrize("prec,arith", [(128, 0), (128, 1), (64, 0)])
def test_30_qubit_workload_plan_invariants(harness, prec, arith):
    # complex64 with the generated kernels' tile cap (2^12), complex128 the default
    head, _ = run(harness, 30, C.workload_30q(), prec=prec, arith=arith, k_req=12 if prec == 64 else 0,
                  emulate=False)
    f = head.split()
    passes, stages = int(f[2]), int(f[4])
    # candidate pass tiles (windows of adjacent qubits) and stages that take
    # later commuting operations: 19 passes, 48 (complex64, R = 5) / 65
    # (complex128, R = 4) stages; the grown tile and in-order stages gave
    # 26-28 passes and 85 / 137 stages
    assert 0 < passes <= 20, head
    assert stages <= (55 if prec == 64 else 75), head


def test_density_matrix_workload_plan_passes(harness):
    """The 14-qubit noisy density-matrix workload: row/column candidate
    tiles keep it at 15 passes (18 with the grown tile alone)."""
    head, _ = run(harness, 14, C.workload_dm14(), density=True, emulate=False)
    assert 0 < int(head.split()[2]) <= 16, head


@pytest.mark.parametrize("p_depol", [0.6, 0.75])
@pytest.mark.parametrize("arith", [0, 1])
def test_planned_density_matrix_heavy_noise(harness, p_depol, arith):
    """Strong channels: the deferred common factor (1 - 2p/3 per
    depolarising channel) passes 2^-30 and is applied mid-plan; p = 3/4
    zeroes the off-diagonal entries (r = 1).  Runs of channels on one qubit
    with only diagonal gates between them share one deferred off-diagonal
    factor."""
    N = 4
    gates = C.random_circuit(N, 8, 500 + int(p_depol * 100), extras=True)
    ops = C.with_noise(gates, 0.3, p_depol)
    extra = [C.Op("T", (1,)), C.Op("CZ", (1, 2)), C.Op("DEPOL", (1,), (), (p_depol,)),
             C.Op("DEPHASE", (1,), (), (0.2,)), C.Op("T", (1,)), C.Op("DEPOL", (1,), (), (0.1,)),
             C.Op("SX", (1,))]
    ops = ops[: len(ops) // 2] + extra + ops[len(ops) // 2:]
    head, rho = run(harness, N, ops, density=True, arith=arith)
    ref = O.run_circuit(N, ops, density=True).a
    assert np.max(np.abs(rho - ref)) <= 1e-12, head


@pytest.mark.parametrize("tile_low", [2, 3, 5])
def test_tile_low_qubits_option_plans_match_oracle(harness, tile_low):
    """Plans whose tiles hold other numbers of contiguous low qubits (the
    "tile_low_qubits" option: shorter HBM chunks, more tile qubits for the
    pass windows) still give the oracle's state: state vectors in both
    precisions and double-float, tiles smaller than the register, noisy
    density matrices."""
    for n, k, prec, arith in ((12, 0, 128, 0), (14, 9, 64, 0), (15, 10, 128, 1), (16, 12, 64, 0)):
        ops = C.random_circuit(n, 12, 500 + n + tile_low, extras=True)
        head, st = run(harness, n, ops, prec=prec, arith=arith, k_req=k, tile_low=tile_low)
        assert np.max(np.abs(st - O.run_circuit(n, ops).a)) <= TOL[(prec, arith)], head
    for N, k, arith in ((5, 8, 0), (6, 0, 1), (6, 10, 0)):
        ops = C.with_noise(C.random_circuit(N, 8, 31 + N, extras=True), 0.05, 0.02)
        head, rho = run(harness, N, ops, density=True, k_req=k, arith=arith, tile_low=tile_low)
        assert np.max(np.abs(rho - O.run_circuit(N, ops, density=True).a)) <= 1e-12, head


def _edge_circuits(n):
    """Shapes at the planner's corners: only diagonal operations (phases,
    CZ, multi-controlled flips: no pass needs a moved bit), every gate on the
    top qubit, alternating top and bottom qubits, a ladder of CNOTs."""
    rng = C.SplitMix64(4000 + n)
    diag = [C.Op(C.H, (q,)) for q in range(n)]
    for i in range(40):
        a, b = C.distinct_qubits(rng, n, 2)
        diag.append([C.Op(C.T_GATE, (a,)), C.Op(C.CZ, (a, b)), C.Op(C.PHASE, (b,), (), (0.1 + rng.uniform(),)),
                     C.Op(C.MCPF, (), tuple(C.distinct_qubits(rng, n, 3)))][i % 4])
    top = [C.Op(C.H, (n - 1,))] + [C.Op([C.SQRT_X, C.SQRT_Y, C.T_GATE][i % 3], (n - 1,)) for i in range(30)]
    alt = [C.Op(C.H, (q,)) for q in range(n)] + \
        [C.Op([C.SQRT_X, C.SQRT_Y][i % 2], ((n - 1) if i % 2 else 0,)) for i in range(30)] + \
        [C.Op(C.CZ, (0, n - 1))]
    ladder = [C.Op(C.H, (0,))] + [C.Op(C.CNOT, (q + 1,), (q,)) for q in range(n - 1)] + \
        [C.Op(C.SQRT_Y, (q,)) for q in range(0, n, 3)]
    return {"diagonal": diag, "top": top, "alternate": alt, "ladder": ladder}


@pytest.mark.parametrize("prec,arith", [(128, 0), (64, 0), (128, 1)])
@pytest.mark.parametrize("n,k", [(13, 0), (14, 13), (16, 10), (18, 12)])
def test_planner_edge_circuits_match_oracle(harness, n, k, prec, arith):
    """The candidate tiles and stage windows on circuits at the planner's
    corners (tile one qubit short of the register, tiles of 2^10 on 16
    qubits, one-tile registers on clusters) still give the oracle's state."""
    for name, ops in _edge_circuits(n).items():
        head, st = run(harness, n, ops, prec=prec, arith=arith, k_req=k)
        err = np.max(np.abs(st - O.run_circuit(n, ops).a))
        assert err <= TOL[(prec, arith)], (name, head, err)


@pytest.mark.parametrize("arith", [0, 1])
def test_planner_density_matrix_channels_only(harness, arith):
    """A density matrix with channels and no gates after a layer of H:
    only deferred off-diagonal factors and diagonal mixes in the passes."""
    N = 6
    ops = [C.Op(C.H, (q,)) for q in range(N)]
    for i in range(24):
        ops.append(C.Op(C.DEPHASE if i % 2 else C.DEPOL, (i % N,), (), (0.02 + 0.01 * (i % 5),)))
    head, rho = run(harness, N, ops, density=True, arith=arith, k_req=8)
    assert np.max(np.abs(rho - O.run_circuit(N, ops, density=True).a)) <= 1e-12, head
