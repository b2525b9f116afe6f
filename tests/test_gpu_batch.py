"""Batched engine (many registers, one graph replay) against the CPU oracle
and against the same registers run alone."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1802_08032_b300 import circuits as C
from gpu_helpers import AMP_TOL, PROB_TOL, fsum_abs2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_1802_08032_b300 import qsim
    return qsim


@pytest.fixture(scope="module")
def env(Q):
    e = Q.createQuESTEnv()
    yield e
    Q.destroyQuESTEnv(e)


def make_regs(Q, env, sizes, prec, seed0, depth=10):
    regs, circs = [], []
    for i, n in enumerate(sizes):
        ops = C.random_circuit(n, depth, seed0 + i, extras=n >= 3)
        q = Q.createQureg(n, prec, env)
        Q.applyCircuit(q, ops)
        regs.append(q)
        circs.append(ops)
    return regs, circs


@pytest.mark.parametrize("prec,arith", [(64, 0), (128, 0), (128, 1)])
def test_batch_matches_oracle(Q, env, prec, arith):
    Q.setEnvOption(env, "arith", arith)
    sizes = [5, 6, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17] * 2
    regs, circs = make_regs(Q, env, sizes, prec, 4096)
    try:
        b = Q.createBatch(env, regs)
        Q.runBatch(b)
        norms = Q.getBatchNorms(b)
        for q, n, ops, nm in zip(regs, sizes, circs, norms):
            got = Q.copyStateToHost(q)
            ref = O.run_circuit(n, ops)
            assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec], n
            assert abs(nm - fsum_abs2(got)) <= PROB_TOL
        # a second replay starts again from |0...0>
        Q.runBatch(b)
        again = Q.getBatchNorms(b)
        assert np.array_equal(again, norms)
        Q.destroyBatch(b)
    finally:
        for q in regs:
            Q.destroyQureg(q)
        Q.setEnvOption(env, "arith", 0)


@pytest.mark.parametrize("prec", [64, 128])
def test_batch_result_equals_alone_bitwise(Q, env, prec):
    """Each register's amplitudes after the batched replay are bit-identical
    to running the same circuit on its own (same planner, same tile size)."""
    sizes = [7, 11, 14, 18, 12, 16]
    regs, circs = make_regs(Q, env, sizes, prec, 777, depth=14)
    try:
        b = Q.createBatch(env, regs, tileQubits=11)
        Q.runBatch(b)
        mixed = [Q.copyStateToHost(q) for q in regs]
        Q.destroyBatch(b)
        Q.setEnvOption(env, "tile_qubits", 11)
        for n, ops, m in zip(sizes, circs, mixed):
            q = Q.createQureg(n, prec, env)
            Q.applyCircuit(q, ops)
            alone = Q.copyStateToHost(q)
            Q.destroyQureg(q)
            assert np.array_equal(alone, m), n
    finally:
        Q.setEnvOption(env, "tile_qubits", 0)
        for q in regs:
            Q.destroyQureg(q)


def test_batch_tuner_and_info(Q, env):
    sizes = [10, 12, 16, 18]
    regs, circs = make_regs(Q, env, sizes, 64, 55)
    try:
        b = Q.createBatch(env, regs)
        info = Q.getBatchInfo(b)
        assert info["waves"] >= 1 and info["passes"] >= len(sizes) and info["bytes"] > 0
        k = Q.tuneBatch(b, [9, 10, 11, 13], replays=1)
        assert k in (9, 10, 11, 13) and Q.getBatchInfo(b)["tileQubits"] == k
        Q.runBatch(b)
        for q, n, ops in zip(regs, sizes, circs):
            ref = O.run_circuit(n, ops)
            assert np.max(np.abs(Q.copyStateToHost(q) - ref.a)) <= AMP_TOL[64]
        Q.destroyBatch(b)
    finally:
        for q in regs:
            Q.destroyQureg(q)


def test_batch_joint_tuner(Q, env):
    """Tile size and fusion depth tuned together: the chosen pair is one of
    the candidates, the batch is re-planned with it (a depth cap of 8 ops
    per pass gives more passes than the default), and every register still
    matches the oracle."""
    sizes = [6, 9, 12, 14, 17]
    regs, circs = make_regs(Q, env, sizes, 64, 56)
    try:
        b = Q.createBatch(env, regs)
        p_default = Q.getBatchInfo(b)["passes"]
        k, d = Q.tuneBatchJoint(b, [8], [8], replays=1)
        assert (k, d) == (8, 8) and Q.getBatchInfo(b)["passes"] > p_default
        k, d = Q.tuneBatchJoint(b, [10, 13], [0, 16, 64], replays=1)
        assert k in (10, 13) and d in (0, 16, 64)
        Q.runBatch(b)
        for q, n, ops in zip(regs, sizes, circs):
            ref = O.run_circuit(n, ops)
            assert np.max(np.abs(Q.copyStateToHost(q) - ref.a)) <= AMP_TOL[64]
        with pytest.raises(Q.QSimError) as e:
            Q.tuneBatchJoint(b, [10], [300])
        assert e.value.name == "QS_E_ARG"
        Q.destroyBatch(b)
    finally:
        for q in regs:
            Q.destroyQureg(q)


def test_batch_argument_errors(Q, env):
    a = Q.createQureg(10, 64, env)
    c = Q.createQureg(10, 128, env)
    d = Q.createDensityQureg(5, 64, env)
    t = Q.createQureg(4, 64, env)
    try:
        for regs, name in (([a, c], "QS_E_ARG"), ([d], "QS_E_ARG"), ([a, a], "QS_E_DUP"),
                           ([t], "QS_E_QUBIT")):
            with pytest.raises(Q.QSimError) as e:
                Q.createBatch(env, regs)
            assert e.value.name == name
        with pytest.raises(Q.QSimError) as e:
            Q.createBatch(env, [a], tileQubits=20)
        assert e.value.name == "QS_E_ARG"
    finally:
        for q in (a, c, d, t):
            Q.destroyQureg(q)
