"""Single-tile fused passes on a thread-block cluster (k_fused_cluster)
against the same passes on one CTA and against the oracle.

A register of at most 13 qubits is one fused tile.  With "fused_cluster" C
its tile is spread over the shared memory of C CTAs, stages whose register
bits include the top log2(C) tile bits read and write the other CTAs'
slices through distributed shared memory, and the rest stay in the CTA's
own slice.  A cluster plan has fewer register bits per stage than the
one-CTA plan, and the planner groups commuting operations into stages by
those bits, so an amplitude may see commuting operations in another order:
the two plans agree to rounding (compared at PLAN_TOL), each is
deterministic (a rerun is bit-identical), and the oracle holds both to the
parity bars."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_1802_08032_b300 import circuits as C
from gpu_helpers import AMP_TOL, PROB_TOL

pytestmark = pytest.mark.gpu

# two plans of one circuit (other stage groupings of commuting operations):
# far below the oracle bars (1e-12 / 1e-5)
PLAN_TOL = {128: 1e-13, 64: 1e-6}


@pytest.fixture(scope="module")
def Q():
    from paper_1802_08032_b300 import qsim
    return qsim


@pytest.fixture(scope="module")
def env(Q):
    e = Q.createQuESTEnv()
    yield e
    Q.destroyQuESTEnv(e)


def run(Q, env, make, ops, cluster, tile=0):
    """The circuit with "fused_cluster" = cluster; tile > 0 fixes the tile
    size (the same plan, one tile, for every cluster size)."""
    Q.setEnvOption(env, "fused_cluster", cluster)
    Q.setEnvOption(env, "tile_qubits", tile)
    try:
        q = make()
        Q.applyCircuit(q, ops)
        tr = Q.calcTotalProb(q)
        got = Q.copyStateToHost(q)
        Q.destroyQureg(q)
    finally:
        Q.setEnvOption(env, "fused_cluster", 8)
        Q.setEnvOption(env, "tile_qubits", 0)
    return got, tr


# registers that are one tile: complex128 tiles hold up to 2^12 amplitudes
# (16 per thread), complex64 up to 2^13 (32 per thread)
SIZES = [(128, 10), (128, 11), (128, 12), (64, 11), (64, 12), (64, 13)]


@pytest.mark.parametrize("prec,n", SIZES)
def test_cluster_state_vector(Q, env, prec, n):
    """Random layers with the extras (controlled and multi-controlled gates,
    phases, general unitaries) on every qubit, so stages put register bits
    on the top tile bits (distributed) and below them (local)."""
    ops = C.random_circuit(n, 16, 700 + n, extras=True)
    make = lambda: Q.createQureg(n, prec, env)  # noqa: E731
    one, tr1 = run(Q, env, make, ops, 0, tile=n)
    for c in (2, 4, 8):
        got, tr = run(Q, env, make, ops, c, tile=n)
        assert np.max(np.abs(got - one)) <= PLAN_TOL[prec], (c, float(np.max(np.abs(got - one))))
        assert abs(tr - tr1) <= (PLAN_TOL[prec] if prec == 128 else 1e-6)
        again, tr_again = run(Q, env, make, ops, c, tile=n)
        assert np.array_equal(again, got) and tr_again == tr
    ref = O.run_circuit(n, ops)
    default, trd = run(Q, env, make, ops, 8)
    for a, t in ((one, tr1), (default, trd)):
        assert np.max(np.abs(a - ref.a)) <= AMP_TOL[prec]
        if prec == 128:
            assert abs(t - ref.total_prob()) <= PROB_TOL


@pytest.mark.parametrize("prec,N", [(128, 5), (128, 6), (64, 6)])
def test_cluster_density_matrix(Q, env, prec, N):
    """Noisy density matrices of 5 and 6 qubits (10- and 12-qubit vectors):
    channels and the conjugated column half of every gate across the
    cluster's slices."""
    ops = C.random_density_circuit(N, 10, 40 + N, 0.01, 0.005)
    make = lambda: Q.createDensityQureg(N, prec, env)  # noqa: E731
    one, tr1 = run(Q, env, make, ops, 0, tile=2 * N)
    for c in (2, 4, 8):
        got, tr = run(Q, env, make, ops, c, tile=2 * N)
        # other stage groupings, and for complex128 the one-CTA plan's 4
        # register bits fold the channels' off-diagonal factors into side
        # operations where the cluster plans' 2-3 do not: equal to rounding
        assert np.max(np.abs(got - one)) <= PLAN_TOL[prec], (c, float(np.max(np.abs(got - one))))
        assert abs(tr - tr1) <= (PLAN_TOL[prec] if prec == 128 else 1e-6)
    ref = O.run_circuit(N, ops, density=True)
    default, trd = run(Q, env, make, ops, 8)
    for a, t in ((one, tr1), (default, trd)):
        assert np.max(np.abs(a - ref.a)) <= AMP_TOL[prec]
        if prec == 128:
            assert abs(t - ref.total_prob()) <= PROB_TOL


def test_cluster_12_qubit_workload(Q, env):
    """The 12-qubit complex128 depth-20 circuit (one tile of 2^12, eight
    CTAs of 32 threads) against the oracle."""
    ops = C.workload_12q()
    one, _ = run(Q, env, lambda: Q.createQureg(12, 128, env), ops, 0, tile=12)
    got, tr = run(Q, env, lambda: Q.createQureg(12, 128, env), ops, 8)
    assert np.max(np.abs(got - one)) <= PLAN_TOL[128]
    ref = O.run_circuit(12, ops)
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[128]
    assert abs(tr - ref.total_prob()) <= PROB_TOL


def test_cluster_option_values(Q, env):
    for v in (0, 1, 2, 4, 8):
        Q.setEnvOption(env, "fused_cluster", v)
        assert Q.getEnvOption(env, "fused_cluster") == v
    for bad in (3, 16, -1):
        with pytest.raises(Q.QSimError) as e:
            Q.setEnvOption(env, "fused_cluster", bad)
        assert e.value.name == "QS_E_ARG"
    Q.setEnvOption(env, "fused_cluster", 8)
