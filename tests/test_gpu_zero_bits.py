"""GPU tests of the known-zero tracking: gates on qubits still in |0> since the
register was zeroed are planned as copies or dropped, so every path that
changes amplitudes must keep that knowledge right.  Each case runs a gate
list through the API paths that touch the tracking and compares the final
state with the oracle."""
import numpy as np
import pytest

from paper_1802_08032_b300 import circuits as C
from oracle import oracle as O
from gpu_helpers import AMP_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_1802_08032_b300 import qsim
    return qsim


@pytest.fixture
def env(Q):
    e = Q.createQuESTEnv()
    yield e
    Q.destroyQuESTEnv(e)


def rand_state(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return a / np.linalg.norm(a)


FIRST = [C.Op("T", (2,)), C.Op("CZ", (1, 3)), C.Op("H", (1,)), C.Op("SX", (4,)), C.Op("SY", (0,)),
         C.Op("MCPF", (), (0, 5, 6)), C.Op("T", (4,)), C.Op("CNOT", (6,), (1,)), C.Op("H", (6,))]


@pytest.mark.parametrize("prec", [128, 64])
def test_fresh_register(Q, env, prec):
    n = 9
    q = Q.createQureg(n, prec, env)
    Q.applyCircuit(q, FIRST)
    got = Q.copyStateToHost(q)
    Q.destroyQureg(q)
    assert np.max(np.abs(got - O.run_circuit(n, FIRST).a)) <= AMP_TOL[prec]


@pytest.mark.parametrize("prec", [128, 64])
def test_after_setamps_and_plus_state(Q, env, prec):
    n = 9
    q = Q.createQureg(n, prec, env)
    psi = rand_state(n, 3)
    Q.setAmps(q, psi)
    Q.applyCircuit(q, FIRST)
    got = Q.copyStateToHost(q)
    ref = O.State(n, amps=psi).run(FIRST).a
    assert np.max(np.abs(got - ref)) <= AMP_TOL[prec]
    Q.initPlusState(q)
    Q.applyCircuit(q, FIRST)
    got = Q.copyStateToHost(q)
    ref = O.State(n, amps=np.full(1 << n, 2 ** (-n / 2), dtype=np.complex128)).run(FIRST).a
    Q.destroyQureg(q)
    assert np.max(np.abs(got - ref)) <= AMP_TOL[prec]


def test_unfused_then_fused(Q, env):
    n = 9
    q = Q.createQureg(n, 128, env)
    Q.setEnvOption(env, "fusion", 0)
    Q.hadamard(q, 2)
    Q.sqrtX(q, 5)
    Q.setEnvOption(env, "fusion", 1)
    ops = [C.Op("H", (2,)), C.Op("T", (5,)), C.Op("H", (5,)), C.Op("CZ", (2, 5))] + FIRST
    Q.applyCircuit(q, ops)
    got = Q.copyStateToHost(q)
    Q.destroyQureg(q)
    ref = O.run_circuit(n, [C.Op("H", (2,)), C.Op("SX", (5,))] + ops).a
    assert np.max(np.abs(got - ref)) <= AMP_TOL[128]


def test_multi_target_on_fresh_qubits(Q, env):
    n = 8
    rng = np.random.default_rng(5)
    m = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    U, _ = np.linalg.qr(m)
    q = Q.createQureg(n, 128, env)
    Q.hadamard(q, 0)
    Q.twoQubitUnitary(q, 3, 6, U)
    Q.applyCircuit(q, [C.Op("H", (3,)), C.Op("T", (6,)), C.Op("SX", (6,)), C.Op("H", (7,))])
    got = Q.copyStateToHost(q)
    Q.destroyQureg(q)
    ref = O.State(n)
    ref.gate(0, O.MAT_H)
    ref.multi((3, 6), U)
    ref.run([C.Op("H", (3,)), C.Op("T", (6,)), C.Op("SX", (6,)), C.Op("H", (7,))])
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[128]


def test_collapse_then_gates_and_rezero(Q, env):
    n = 7
    q = Q.createQureg(n, 128, env)
    ref = O.State(n)
    pre = [C.Op("H", (0,)), C.Op("CNOT", (1,), (0,))]
    Q.applyCircuit(q, pre)
    ref.run(pre)
    p = Q.collapseToOutcome(q, 1, 1)
    assert abs(p - ref.collapse(1, 1)) <= 1e-13
    post = [C.Op("H", (4,)), C.Op("T", (1,)), C.Op("SY", (1,)), C.Op("CZ", (0, 4))]
    Q.applyCircuit(q, post)
    ref.run(post)
    assert np.max(np.abs(Q.copyStateToHost(q) - ref.a)) <= AMP_TOL[128]
    Q.initZeroState(q)
    Q.applyCircuit(q, FIRST[:6])
    got = Q.copyStateToHost(q)
    Q.destroyQureg(q)
    assert np.max(np.abs(got - O.run_circuit(n, FIRST[:6]).a)) <= AMP_TOL[128]


def test_density_matrix_fresh_and_after_plus(Q, env):
    N = 4
    ops = C.with_noise([C.Op("T", (1,)), C.Op("H", (1,)), C.Op("SX", (2,)), C.Op("CZ", (1, 2)),
                        C.Op("T", (3,))], 0.02, 0.01)
    d = Q.createDensityQureg(N, 128, env)
    Q.applyCircuit(d, ops)
    got = Q.copyStateToHost(d)
    assert np.max(np.abs(got - O.run_circuit(N, ops, density=True).a)) <= AMP_TOL[128]
    Q.initPlusState(d)
    Q.applyCircuit(d, ops)
    got = Q.copyStateToHost(d)
    Q.destroyQureg(d)
    plus = np.full(1 << (2 * N), 2.0 ** -N, dtype=np.complex128)
    ref = O.State(N, density=True, amps=plus).run(ops).a
    assert np.max(np.abs(got - ref)) <= AMP_TOL[128]


def test_gates_after_batch_replay(Q, env):
    sizes = [6, 9]
    regs = [Q.createQureg(n, 128, env) for n in sizes]
    circs = [C.random_circuit(n, 5, 60 + n, extras=True) for n in sizes]
    try:
        for q, ops in zip(regs, circs):
            Q.applyCircuit(q, ops)
        b = Q.createBatch(env, regs)
        Q.runBatch(b)
        Q.runBatch(b)
        Q.destroyBatch(b)
        more = [C.Op("H", (2,)), C.Op("T", (3,)), C.Op("SX", (3,))]
        for q, n, ops in zip(regs, sizes, circs):
            Q.applyCircuit(q, more)
            got = Q.copyStateToHost(q)
            assert np.max(np.abs(got - O.run_circuit(n, ops + more).a)) <= AMP_TOL[128], n
    finally:
        for q in regs:
            Q.destroyQureg(q)


def test_raw_pointer_clears_tracking(Q, env):
    """A caller may write the amplitudes through getQuregInfo's pointer."""
    rt = pytest.importorskip("cuda.bindings.runtime")
    n = 6
    q = Q.createQureg(n, 128, env)
    ptr = Q.getQuregInfo(q)["devicePtr"]
    Q.syncQuESTEnv(env)
    psi = rand_state(n, 9)
    host = np.ascontiguousarray(psi)  # interleaved (re, im) doubles, the register's layout
    (err,) = rt.cudaMemcpy(ptr, host.ctypes.data, host.nbytes, rt.cudaMemcpyKind.cudaMemcpyHostToDevice)
    assert int(err) == 0
    ops = [C.Op("H", (1,)), C.Op("T", (2,)), C.Op("CZ", (2, 4))]
    Q.applyCircuit(q, ops)
    got = Q.copyStateToHost(q)
    Q.destroyQureg(q)
    assert np.max(np.abs(got - O.State(n, amps=psi).run(ops).a)) <= AMP_TOL[128]


@pytest.mark.parametrize("prec", [128, 64])
@pytest.mark.parametrize("density", [False, True])
def test_unfused_pending_scale(Q, env, prec, density):
    """Unfused uncontrolled H / sqrt(X) / sqrt(Y) passes leave their scalar
    factors to the register; reductions, collapse, copies and a later fused
    flush must all see the scaled values, and 600 such passes (float range:
    the factor is settled before it underflows) stay finite."""
    n = 3 if density else 8
    rng = C.SplitMix64(600 + prec + density)
    kinds = ("H", "SX", "SY", "T", "CZ")
    ops = []
    for _ in range(600):
        k = kinds[rng.below(5)]
        if k == "CZ":
            a, b = C.distinct_qubits(rng, n, 2)
            ops.append(C.Op("CZ", (a, b)))
        else:
            ops.append(C.Op(k, (rng.below(n),)))
    Q.setEnvOption(env, "fusion", 0)
    try:
        q = (Q.createDensityQureg if density else Q.createQureg)(n, prec, env)
        ref = O.State(n, density=density)
        Q.applyCircuit(q, ops[:300])
        ref.run(ops[:300])
        tol = 1e-12 if prec == 128 else 1e-5
        assert abs(Q.calcTotalProb(q) - ref.total_prob()) <= tol
        assert abs(Q.calcProbOfOutcome(q, 1, 0) - ref.prob_outcome(1, 0)) <= tol
        if density:
            assert abs(Q.calcPurity(q) - ref.purity()) <= tol
        Q.applyCircuit(q, ops[300:450])
        ref.run(ops[300:450])
        p = Q.collapseToOutcome(q, 0, 1)
        assert abs(p - ref.collapse(0, 1)) <= (1e-12 if prec == 128 else 1e-5)
        Q.applyCircuit(q, ops[450:])
        ref.run(ops[450:])
        got = Q.copyStateToHost(q)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec] * (10 if prec == 64 else 1)
        Q.setEnvOption(env, "fusion", 1)
        more = [C.Op("SX", (1,)), C.Op("T", (2,)), C.Op("H", (0,))]
        Q.hadamard(q, 1)  # queued again: fused with `more` at the next copy
        ref.gate(1, O.MAT_H)
        Q.applyCircuit(q, more)
        ref.run(more)
        got = Q.copyStateToHost(q)
        Q.destroyQureg(q)
        assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec] * (10 if prec == 64 else 1)
    finally:
        Q.setEnvOption(env, "fusion", 1)


def test_unfused_phase_factor_per_qubit(Q, env):
    """Unfused complex128 phases run as 1 + i tan(phi) and leave cos(phi) as a
    factor on the qubit's bit-1 half: the next uncontrolled H / sqrt(X) /
    sqrt(Y) on the qubit takes it, a general, controlled or multi-target
    update on the qubit and every read apply it first, gates that only use
    the qubit as a control or are diagonal leave it pending."""
    n = 9
    rng = np.random.default_rng(12)
    m = rng.normal(size=(8, 8)) + 1j * rng.normal(size=(8, 8))
    U3, _ = np.linalg.qr(m)
    a = complex(0.6, 0.0)
    b = complex(0.0, 0.8)
    seq = [
        [C.Op("T", (1,)), C.Op("T", (1,)), C.Op("T", (1,)), C.Op("SX", (1,))],        # taken by sqrt(X)
        [C.Op("T", (2,)), C.Op("CNOT", (5,), (2,)), C.Op("CZ", (2, 3)), C.Op("H", (2,))],  # control, diagonal, then H
        [C.Op("T", (3,)), C.Op("COMPACT", (3,), (), (a.real, a.imag, b.real, b.imag))],  # general: applied first
        [C.Op("T", (4,)), C.Op("CUNITARY", (4,), (0,), (0.6, 0, 0, -0.8, 0, -0.8, 0.6, 0))],  # controlled update on it
        [C.Op("T", (6,)), C.Op("PHASE", (6,), (), (0.7,)), C.Op("SY", (6,))],
        [C.Op("T", (7,))] * 5 + [C.Op("T", (0,))],                                      # left pending until the read
    ]
    Q.setEnvOption(env, "fusion", 0)
    try:
        q = Q.createQureg(n, 128, env)
        ref = O.State(n)
        for ops in seq:
            Q.applyCircuit(q, ops)
            ref.run(ops)
        Q.multiControlledMultiQubitUnitary(q, (), (7, 8, 0), U3)  # targets with pending factors
        ref.multi((7, 8, 0), U3)
        Q.applyCircuit(q, [C.Op("T", (5,)), C.Op("T", (8,))])
        ref.run([C.Op("T", (5,)), C.Op("T", (8,))])
        assert abs(Q.calcProbOfOutcome(q, 5, 1) - ref.prob_outcome(5, 1)) <= 1e-13
        Q.applyCircuit(q, [C.Op("T", (5,))] * 400 + [C.Op("H", (5,))])  # the factor is bounded
        ref.run([C.Op("T", (5,))] * 400 + [C.Op("H", (5,))])
        p = Q.collapseToOutcome(q, 8, 0)
        assert abs(p - ref.collapse(8, 0)) <= 1e-13
        Q.applyCircuit(q, [C.Op("T", (2,))])
        ref.run([C.Op("T", (2,))])
        Q.setEnvOption(env, "fusion", 1)  # queued from here: the flush plans with the factors applied
        more = [C.Op("SX", (2,)), C.Op("T", (6,)), C.Op("CZ", (2, 6)), C.Op("H", (6,))]
        Q.applyCircuit(q, more)
        ref.run(more)
        got = Q.copyStateToHost(q)
        Q.destroyQureg(q)
        assert np.max(np.abs(got - ref.a)) <= AMP_TOL[128]
    finally:
        Q.setEnvOption(env, "fusion", 1)


def test_unfused_general_updates_phase_shear(Q, env):
    """Unfused complex128 uncontrolled general updates run as phase-shear:
    the qubit's pending factor folds into the matrix, the output phase stays
    pending.  Chains of general updates, H / sqrt(X) / sqrt(Y) meeting a
    complex pending factor, X, controlled and multi-target updates that apply
    it first, uses as a control, reads, and a switch back to fused flushes."""
    n = 8
    rng = C.SplitMix64(77)

    def haar():
        a = C.haar_alpha_beta(rng)
        return C.Op("COMPACT", (rng.below(n),), (), tuple(a))

    ops = []
    for _ in range(120):
        k = rng.below(8)
        q = rng.below(n)
        if k <= 2:
            ops.append(haar())
        elif k == 3:
            ops.append(C.Op(("H", "SX", "SY")[rng.below(3)], (q,)))
        elif k == 4:
            ops.append(C.Op("T", (q,)))
        elif k == 5:
            c = (q + 1 + rng.below(n - 1)) % n
            ops.append(C.Op("CNOT", (q,), (c,)))
        elif k == 6:
            ops.append(C.Op("X", (q,)))
        else:
            a, b = C.distinct_qubits(rng, n, 2)
            ops.append(C.Op("CZ", (a, b)))
    same = C.Op("COMPACT", (3,), (), tuple(C.haar_alpha_beta(rng)))
    chain = [same] * 300 + [C.Op("SX", (3,)), C.Op("H", (3,))]
    g = np.random.default_rng(4)
    U2 = np.linalg.qr(g.normal(size=(4, 4)) + 1j * g.normal(size=(4, 4)))[0]
    Q.setEnvOption(env, "fusion", 0)
    try:
        q = Q.createQureg(n, 128, env)
        ref = O.State(n)
        Q.applyCircuit(q, ops[:60])
        ref.run(ops[:60])
        assert abs(Q.calcTotalProb(q) - 1.0) <= 1e-13
        Q.applyCircuit(q, ops[60:] + chain)
        ref.run(ops[60:] + chain)
        Q.applyCircuit(q, [same, C.Op("T", (3,)), same])
        ref.run([same, C.Op("T", (3,)), same])
        Q.multiControlledMultiQubitUnitary(q, (5,), (3, 0), U2)
        ref.multi((3, 0), U2, (5,))
        assert abs(Q.calcProbOfOutcome(q, 3, 1) - ref.prob_outcome(3, 1)) <= 1e-13
        Q.applyCircuit(q, [same, C.Op("CNOT", (1,), (3,))])
        ref.run([same, C.Op("CNOT", (1,), (3,))])
        Q.setEnvOption(env, "fusion", 1)
        tail = [C.Op("SY", (3,)), C.Op("T", (1,)), C.Op("CZ", (1, 3))]
        Q.applyCircuit(q, tail)
        ref.run(tail)
        got = Q.copyStateToHost(q)
        Q.destroyQureg(q)
        assert np.max(np.abs(got - ref.a)) <= AMP_TOL[128]
    finally:
        Q.setEnvOption(env, "fusion", 1)
