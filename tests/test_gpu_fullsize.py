"""Full-size parity: the GPU path at the benchmark configurations' sizes
against expected values the CPU oracle wrote (tests/golden/make_golden.py):
sampled amplitudes, reductions and outcome probabilities."""
import json
import os

import numpy as np
import pytest

from paper_1802_08032_b300 import circuits as C
from gpu_helpers import AMP_TOL, PROB_TOL, inverse

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated yet")
    with open(path) as f:
        return json.load(f)


def as_complex(pairs):
    a = np.array(pairs, dtype=np.float64)
    return a[:, 0] + 1j * a[:, 1]


@pytest.fixture(scope="module")
def Q():
    from paper_1802_08032_b300 import qsim
    return qsim


@pytest.fixture(scope="module")
def env(Q):
    e = Q.createQuESTEnv()
    yield e
    Q.destroyQuESTEnv(e)


def sample(Q, q, idx):
    return np.array([Q.copyStateToHost(q, int(i), 1)[0] for i in idx])


@pytest.mark.parametrize("arith", [0, 1])
def test_density_matrix_14_qubits(Q, env, arith):
    g = golden("dm14_depth20.json")
    ops = C.workload_dm14(14)
    assert C.stream_hash(ops) == g["hash"]
    Q.setEnvOption(env, "arith", arith)
    try:
        d = Q.createDensityQureg(14, 128, env)
        Q.applyCircuit(d, ops)
        tr, pur = Q.calcTotalProb(d), Q.calcPurity(d)
        probs = [Q.calcProbOfOutcome(d, q, 1) for q in range(14)]
        got = sample(Q, d, g["indices"])
        n = 1 << 14
        diag = sample(Q, d, [j + n * j for j in g["diag_rows"]])
        Q.destroyQureg(d)
    finally:
        Q.setEnvOption(env, "arith", 0)
    assert abs(tr - g["trace"]) <= PROB_TOL
    assert abs(pur - g["purity"]) <= PROB_TOL
    assert np.max(np.abs(np.array(probs) - g["prob_outcome_1"])) <= PROB_TOL
    assert np.max(np.abs(got - as_complex(g["amps"]))) <= AMP_TOL[128]
    assert np.max(np.abs(diag - as_complex(g["diag"]))) <= AMP_TOL[128]


def shifted(ops, k):
    return [C.Op(o.kind, tuple(t + k for t in o.targets), tuple(c + k for c in o.controls), o.params)
            for o in ops]


@pytest.mark.parametrize("prec,arith", [(128, 0), (128, 1), (64, 0)])
def test_33_qubit_product_state(Q, env, prec, arith):
    """33 qubits (2^33 amplitudes: 128 GiB complex128, 64 GiB complex64): a
    30-qubit circuit on qubits 0..29 and a 3-qubit circuit on 30..32; every
    sampled amplitude is the product of the two factors' amplitudes (64-bit
    indices throughout).  Runs the IEEE-FP64 and complex64 fused kernels as
    well as the double-float one."""
    g = golden("sv33_product_factors.json")
    low = C.random_circuit(30, 12, 3330, extras=True)
    high = C.random_circuit(3, 12, 3333, extras=True)
    assert C.stream_hash(low) == g["hash_low"] and C.stream_hash(high) == g["hash_high"]
    Q.setEnvOption(env, "arith", arith)
    try:
        q = Q.createQureg(33, prec, env)
        Q.applyCircuit(q, low + shifted(high, 30))
        tot = Q.calcTotalProb(q)
        probs_hi = [Q.calcProbOfOutcome(q, 30 + k, 1) for k in range(3)]
        probs_lo = [Q.calcProbOfOutcome(q, k, 1) for k in (0, 13, 29)]
        lo_idx = g["low_indices"][:512]
        lo_amp = as_complex(g["low_amps"])[:512]
        hi_amp = as_complex(g["high_amps"])
        idx = [(j << 30) + i for j in range(8) for i in lo_idx]
        got = sample(Q, q, idx)
        Q.destroyQureg(q)
    finally:
        Q.setEnvOption(env, "arith", 0)
    want = np.array([hi_amp[j] * a for j in range(8) for a in lo_amp])
    assert np.max(np.abs(got - want)) <= AMP_TOL[prec]
    tol = PROB_TOL if prec == 128 else 1e-5
    assert abs(tot - g["low_total_prob"]) <= tol
    assert np.max(np.abs(np.array(probs_hi) - g["high_prob_outcome_1"])) <= tol
    assert np.max(np.abs(np.array(probs_lo) - np.array(g["low_prob_outcome_1"])[[0, 13, 29]])) <= tol


@pytest.mark.parametrize("prec", [128, 64])
def test_33_qubit_mirror_circuit(Q, env, prec):
    """33-qubit depth-40 workload C followed by C-dagger returns |0...0>
    (no host oracle: the 128 GiB state does not fit a host).  Pins the
    full-size 64-bit index paths of the fused kernels (IEEE FP64 and
    complex64) by a closed form."""
    ops = C.workload_30q(33)
    q = Q.createQureg(33, prec, env)
    try:
        Q.applyCircuit(q, ops + inverse(ops))
        tot = Q.calcTotalProb(q)
        probs = [Q.calcProbOfOutcome(q, k, 1) for k in range(33)]
        head = Q.copyStateToHost(q, 0, 64)
        tail = Q.copyStateToHost(q, (1 << 33) - 64, 64)
    finally:
        Q.destroyQureg(q)
    tol = AMP_TOL[prec]
    assert abs(head[0] - 1) <= tol
    assert np.max(np.abs(head[1:])) <= tol and np.max(np.abs(tail)) <= tol
    # No oracle runs here, so the bar is the closed form's own rounding
    # budget: every one of the 2756 gate applications may change the norm by
    # a few units in the last place (at most 4 u, u = 2^-53 for FP64), which
    # an exact-rounding implementation would show too (FP64 measured:
    # |1 - total| = 1.6e-13).  The amplitude bars above are the stated ones.
    ptol = len(ops) * 2 * 4 * 2.0 ** -53 if prec == 128 else 1e-5
    assert abs(tot - 1) <= ptol
    assert max(probs) <= ptol


@pytest.mark.parametrize("prec,arith", [(128, 0), (128, 1), (64, 0)])
def test_30_qubit_depth40_workload(Q, env, prec, arith):
    g = golden("sv30_depth40.json")
    ops = C.workload_30q(30)
    assert C.stream_hash(ops) == g["hash"]
    Q.setEnvOption(env, "arith", arith)
    try:
        q = Q.createQureg(30, prec, env)
        Q.applyCircuit(q, ops)
        tot = Q.calcTotalProb(q)
        probs = [Q.calcProbOfOutcome(q, k, 1) for k in range(30)]
        got = sample(Q, q, g["indices"])
        Q.destroyQureg(q)
    finally:
        Q.setEnvOption(env, "arith", 0)
    assert np.max(np.abs(got - as_complex(g["amps"]))) <= AMP_TOL[prec]
    # Double-float (an out-of-spec precision form: 48-bit significands, a few
    # units of 2^-48 per update) is held to the complex128 bar as well: with
    # 19 passes (each pass boundary rounds the float pairs to doubles) its
    # FP64-reduced probabilities stay within 6e-14 of the oracle here.
    tol = PROB_TOL if prec == 128 else 1e-5
    assert abs(tot - g["total_prob"]) <= tol
    assert np.max(np.abs(np.array(probs) - g["prob_outcome_1"])) <= tol


@pytest.mark.parametrize("prec", [128, 64])
def test_30_qubit_depth40_workload_unfused(Q, env, prec):
    """The same 30-qubit circuit one kernel per gate: unscaled H / sqrt(X) /
    sqrt(Y) with the register's scalar, (1 + i tan) phases and phase-shear
    general updates with per-qubit factors, at full size."""
    g = golden("sv30_depth40.json")
    ops = C.workload_30q(30)
    Q.setEnvOption(env, "fusion", 0)
    try:
        q = Q.createQureg(30, prec, env)
        Q.applyCircuit(q, ops)
        tot = Q.calcTotalProb(q)
        probs = [Q.calcProbOfOutcome(q, k, 1) for k in range(0, 30, 3)]
        got = sample(Q, q, g["indices"])
        Q.destroyQureg(q)
    finally:
        Q.setEnvOption(env, "fusion", 1)
    assert np.max(np.abs(got - as_complex(g["amps"]))) <= AMP_TOL[prec]
    tol = PROB_TOL if prec == 128 else 1e-5
    assert abs(tot - g["total_prob"]) <= tol
    assert np.max(np.abs(np.array(probs) - np.array(g["prob_outcome_1"])[0:30:3])) <= tol
