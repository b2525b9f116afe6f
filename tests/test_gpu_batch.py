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


@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("prec,arith", [(64, 0), (128, 0), (128, 1)])
def test_batch_matches_oracle(Q, env, prec, arith, persistent):
    Q.setEnvOption(env, "arith", arith)
    Q.setEnvOption(env, "batch_persistent", persistent)
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
        Q.setEnvOption(env, "batch_persistent", 1)


@pytest.mark.parametrize("prec", [64, 128])
def test_persistent_batch_equals_wave_launches_bitwise(Q, env, prec):
    """The persistent form (one launch; CTAs claim items in wave order and
    wait for a register's previous pass) gives the amplitudes of the
    one-launch-per-wave graph bit for bit: the same tiles with the same
    arithmetic, only scheduled differently.  Many registers with several
    passes each, so passes of different registers overlap; two replays."""
    rng = C.SplitMix64(2024)
    sizes = [8 + rng.below(11) for _ in range(160)]
    regs, circs = make_regs(Q, env, sizes, prec, 9000, depth=16)
    out = {}
    try:
        for persistent in (0, 1):
            Q.setEnvOption(env, "batch_persistent", persistent)
            if persistent:   # the first batch took the registers' queued gates
                for q, ops in zip(regs, circs):
                    Q.applyCircuit(q, ops)
            b = Q.createBatch(env, regs, tileQubits=10)
            assert Q.getBatchInfo(b)["waves"] >= 3
            states = []
            for _ in range(2):
                Q.runBatch(b)
                norms = Q.getBatchNorms(b)
                states.append([Q.copyStateToHost(q) for q in regs])
            for x, y in zip(*states):
                assert np.array_equal(x, y)
            out[persistent] = (states[0], norms)
            Q.destroyBatch(b)
        for n, x, y in zip(sizes, out[0][0], out[1][0]):
            assert np.array_equal(x, y), n
        assert np.array_equal(out[0][1], out[1][1])
        for i in range(0, len(sizes), 23):
            ref = O.run_circuit(sizes[i], circs[i])
            assert np.max(np.abs(out[1][0][i] - ref.a)) <= AMP_TOL[prec]
    finally:
        Q.setEnvOption(env, "batch_persistent", 1)
        for q in regs:
            Q.destroyQureg(q)


@pytest.mark.parametrize("prec", [64, 128])
def test_batch_result_equals_alone_bitwise(Q, env, prec):
    """Each register's amplitudes after the batched replay are bit-identical
    to running the same circuit on its own (same planner, same tile size;
    one CTA per tile, as in the batch: a thread-block cluster plan groups
    its stages by fewer register bits)."""
    sizes = [7, 11, 14, 18, 12, 16]
    regs, circs = make_regs(Q, env, sizes, prec, 777, depth=14)
    try:
        b = Q.createBatch(env, regs, tileQubits=11)
        Q.runBatch(b)
        mixed = [Q.copyStateToHost(q) for q in regs]
        Q.destroyBatch(b)
        Q.setEnvOption(env, "tile_qubits", 11)
        Q.setEnvOption(env, "fused_cluster", 0)
        for n, ops, m in zip(sizes, circs, mixed):
            q = Q.createQureg(n, prec, env)
            Q.applyCircuit(q, ops)
            alone = Q.copyStateToHost(q)
            Q.destroyQureg(q)
            assert np.array_equal(alone, m), n
    finally:
        Q.setEnvOption(env, "tile_qubits", 0)
        Q.setEnvOption(env, "fused_cluster", 8)
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


@pytest.mark.parametrize("persistent", [0, 1])
def test_batch_of_registers_without_gates(Q, env, persistent):
    """Registers with nothing queued: the replay launches no pass (and the
    persistent form no empty launch) and every register reads |0...0>."""
    Q.setEnvOption(env, "batch_persistent", persistent)
    regs = [Q.createQureg(n, 64, env) for n in (6, 9, 12)]
    try:
        b = Q.createBatch(env, regs)
        Q.runBatch(b)
        assert np.array_equal(Q.getBatchNorms(b), np.ones(3))
        for q in regs:
            a = Q.copyStateToHost(q)
            assert a[0] == 1 and not np.any(a[1:])
        Q.destroyBatch(b)
    finally:
        Q.setEnvOption(env, "batch_persistent", 1)
        for q in regs:
            Q.destroyQureg(q)


def test_persistent_batch_bounded_wait_reports_timeout(Q, env):
    """The persistent form's wait for a register's previous pass is bounded:
    with every dependency one tile short (diagnostic option, 2 ms bound) the
    wait runs out, the launch ends, getBatchNorms reports QS_E_TIMEOUT once,
    and the context keeps working (a normal batch afterwards matches the
    oracle).  No fault and no unbounded wait."""
    sizes = [12, 15, 17]
    regs, circs = make_regs(Q, env, sizes, 64, 71, depth=12)
    try:
        Q.setEnvOption(env, "batch_diag_stall", 1)
        b = Q.createBatch(env, regs, tileQubits=10)
        Q.setEnvOption(env, "batch_diag_stall", 0)
        assert Q.getBatchInfo(b)["waves"] >= 2
        Q.runBatch(b)
        with pytest.raises(Q.QSimError) as e:
            Q.getBatchNorms(b)
        assert e.value.name == "QS_E_TIMEOUT"
        Q.destroyBatch(b)
        Q.syncQuESTEnv(env)   # the status word was cleared: no second report
        for q, ops in zip(regs, circs):
            Q.applyCircuit(q, ops)
        b = Q.createBatch(env, regs, tileQubits=10)
        Q.runBatch(b)
        Q.getBatchNorms(b)
        for q, n, ops in zip(regs, sizes, circs):
            ref = O.run_circuit(n, ops)
            assert np.max(np.abs(Q.copyStateToHost(q) - ref.a)) <= AMP_TOL[64]
        Q.destroyBatch(b)
    finally:
        Q.setEnvOption(env, "batch_diag_stall", 0)
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
