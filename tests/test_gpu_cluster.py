"""Single-tile fused passes on a thread-block cluster (k_fused_cluster)
against the same passes on one CTA and against the oracle.

A register of at most 13 qubits is one fused tile.  With "fused_cluster" C
its tile is spread over the shared memory of C CTAs, stages whose register
bits include the top log2(C) tile bits read and write the other CTAs'
slices through distributed shared memory, and the rest stay in the CTA's
own slice.  Every amplitude sees the same operations in the same order as on
one CTA, so the results are compared bit for bit; the oracle holds both to
the parity bars."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1802_08032_b300 import circuits as C
from gpu_helpers import AMP_TOL, PROB_TOL

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
        assert np.array_equal(got, one), (c, float(np.max(np.abs(got - one))))
        assert tr == tr1
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
        if prec == 64:
            assert np.array_equal(got, one), (c, float(np.max(np.abs(got - one))))
            assert tr == tr1
        else:
            # complex128 density plans with 4 register bits (one CTA) fold
            # the channels' off-diagonal factors into side operations, the
            # cluster plans' 2-3 register bits do not: the same products in
            # another order, equal to rounding
            assert np.max(np.abs(got - one)) <= 1e-15, c
            assert abs(tr - tr1) <= 1e-15
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
    assert np.array_equal(got, one)
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
