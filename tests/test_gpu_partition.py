"""Partitioned state vectors on the GPU: 2^k parts with qubit swaps through
send / receive buffers (the paper's distributed scheme, Sec. II.B.2, with
every part on this GPU) against the oracle's full state."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1802_08032_b300 import circuits as C
from gpu_helpers import AMP_TOL, PROB_TOL
from test_partition_cpu import circuit

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


@pytest.mark.parametrize("fusion", [1, 0])
@pytest.mark.parametrize("prec", [128, 64])
@pytest.mark.parametrize("n,k", [(8, 1), (12, 2), (14, 3)])
def test_partitioned_register_matches_oracle(Q, env, n, k, prec, fusion):
    ops = circuit(n, 300 + n)
    Q.setEnvOption(env, "fusion", fusion)
    r = Q.createPartitionedQureg(n, k, prec, env)
    try:
        # two calls: the qubit map and the parts carry over between them
        Q.partApplyCircuit(r, ops[: len(ops) // 2])
        Q.partApplyCircuit(r, ops[len(ops) // 2:])
        got = Q.partCopyStateToHost(r)
        tot = Q.partCalcTotalProb(r)
        probs = [Q.partCalcProbOfOutcome(r, q, 1) for q in range(n)]
        info = Q.partGetInfo(r)
    finally:
        Q.destroyPartitionedQureg(r)
        Q.setEnvOption(env, "fusion", 1)
    ref = O.run_circuit(n, ops)
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec]
    ptol = PROB_TOL if prec == 128 else 1e-5
    assert abs(tot - ref.total_prob()) <= ptol
    assert max(abs(p - ref.prob_outcome(q, 1)) for q, p in enumerate(probs)) <= ptol
    assert info["swaps"] > 0 and info["exchangedBytes"] > 0
    assert sorted(info["perm"]) == list(range(n))
    steps, perm = Q.partPlanSchedule(n, k, ops)
    assert info["swaps"] >= sum(1 for s in steps if s[0] == 1) - 1  # (split in two calls)


def test_partitioned_register_30_ops_per_layer_workload(Q, env):
    """The 16-qubit depth-20 workload layering over 4 parts, complex128."""
    n, k = 16, 2
    ops = C.workload_30q(n)[:400]
    r = Q.createPartitionedQureg(n, k, 128, env)
    try:
        Q.partApplyCircuit(r, ops)
        got = Q.partCopyStateToHost(r)
    finally:
        Q.destroyPartitionedQureg(r)
    assert np.max(np.abs(got - O.run_circuit(n, ops).a)) <= AMP_TOL[128]


def test_partitioned_register_errors(Q, env):
    for n, k in ((1, 1), (8, 0), (8, 8), (10, 7)):
        with pytest.raises(Q.QSimError) as e:
            Q.createPartitionedQureg(n, k, 128, env)
        assert e.value.name == "QS_E_QUBIT"
    r = Q.createPartitionedQureg(6, 2, 128, env)
    try:
        with pytest.raises(Q.QSimError) as e:
            Q.partApplyCircuit(r, [C.Op("DEPHASE", (1,), (), (0.1,))])
        assert e.value.name == "QS_E_NOT_DENSITY"
        with pytest.raises(Q.QSimError) as e:
            Q.partApplyCircuit(r, [C.Op("H", (6,))])
        assert e.value.name == "QS_E_QUBIT"
        with pytest.raises(Q.QSimError) as e:
            Q.partCalcProbOfOutcome(r, 0, 2)
        assert e.value.name == "QS_E_PROB"
        # the register is unchanged by the refused calls
        assert abs(Q.partCopyStateToHost(r)[0] - 1) == 0
    finally:
        Q.destroyPartitionedQureg(r)
