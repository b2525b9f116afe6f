"""GPU path vs the CPU oracle, element by element, through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1802_08032_b300 import circuits as C
from gpu_helpers import (AMP_TOL, PROB_TOL, fsum_abs2, gpu_state, rand_density_vec, rand_state,
                         single_ops)

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


@pytest.mark.parametrize("prec", [128, 64])
@pytest.mark.parametrize("fusion", [0, 1])
def test_every_gate_every_target(Q, env, prec, fusion):
    n = 9
    psi = rand_state(n, 11)
    for op in single_ops(n, seed=3):
        ref = O.State(n, amps=psi)
        ref.apply(op)
        got = gpu_state(Q, env, n, [op], prec, fusion=fusion, init=psi)
        err = np.max(np.abs(got - ref.a))
        assert err <= AMP_TOL[prec] * (1 if prec == 128 else 0.1), (op, err)


@pytest.mark.parametrize("prec", [128, 64])
@pytest.mark.parametrize("fusion", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11, 14])
def test_random_circuits(Q, env, prec, fusion, n):
    ops = C.random_circuit(n, 12, 100 + n, extras=n >= 3)
    ref = O.run_circuit(n, ops)
    got = gpu_state(Q, env, n, ops, prec, fusion=fusion)
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec]


@pytest.mark.parametrize("prec", [128, 64])
def test_twelve_qubit_depth20_workload(Q, env, prec):
    """12-qubit state vector, depth-20 random circuit, then calcTotalProb and
    calcProbOfOutcome on qubit 0."""
    ops = C.workload_12q()
    ref = O.run_circuit(12, ops)
    Q.setEnvOption(env, "fusion", 1)
    q = Q.createQureg(12, prec, env)
    Q.applyCircuit(q, ops)
    tot = Q.calcTotalProb(q)
    p0, p1 = Q.calcProbOfOutcome(q, 0, 0), Q.calcProbOfOutcome(q, 0, 1)
    got = Q.copyStateToHost(q)
    Q.destroyQureg(q)
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec]
    if prec == 128:
        assert abs(tot - ref.total_prob()) <= PROB_TOL
        assert abs(p0 - ref.prob_outcome(0, 0)) <= PROB_TOL
        assert abs(p1 - ref.prob_outcome(0, 1)) <= PROB_TOL
    else:
        # FP64 reduction of the GPU's own complex64 amplitudes
        assert abs(tot - fsum_abs2(got)) <= PROB_TOL
        sel = (np.arange(got.size) & 1) == 0
        assert abs(p0 - fsum_abs2(got[sel])) <= PROB_TOL
        assert abs(p0 - ref.prob_outcome(0, 0)) <= 1e-5


@pytest.mark.parametrize("prec", [128, 64])
def test_twenty_qubit_circuit(Q, env, prec):
    ops = C.random_circuit(20, 16, 2020, extras=True)
    ref = O.run_circuit(20, ops)
    got = gpu_state(Q, env, 20, ops, prec)
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec]


# ----------------------------------------------------------- density matrix
@pytest.mark.parametrize("prec", [128, 64])
@pytest.mark.parametrize("fusion", [0, 1])
def test_density_every_gate_and_channel(Q, env, prec, fusion):
    N = 4
    rho = rand_density_vec(N, 5)
    ops = single_ops(N, seed=9)
    for t in range(N):
        ops += [C.Op("DEPHASE", (t,), (), (0.13,)), C.Op("DEPOL", (t,), (), (0.21,)),
                C.Op("PHASE", (t,), (), (0.7,))]
    for op in ops:
        ref = O.State(N, density=True, amps=rho)
        ref.apply(op)
        got = gpu_state(Q, env, N, [op], prec, density=True, fusion=fusion, init=rho)
        err = np.max(np.abs(got - ref.a))
        assert err <= AMP_TOL[prec] * (1 if prec == 128 else 0.1), (op, err)


@pytest.mark.parametrize("prec", [128, 64])
@pytest.mark.parametrize("fusion", [0, 1])
@pytest.mark.parametrize("N", [1, 3, 6])
def test_noisy_density_circuit(Q, env, prec, fusion, N):
    ops = C.random_density_circuit(N, 10, 14 + N, 0.01, 0.005)
    ref = O.run_circuit(N, ops, density=True)
    Q.setEnvOption(env, "fusion", fusion)
    q = Q.createDensityQureg(N, prec, env)
    Q.applyCircuit(q, ops)
    tr, pur = Q.calcTotalProb(q), Q.calcPurity(q)
    probs = [Q.calcProbOfOutcome(q, t, 1) for t in range(N)]
    got = Q.copyStateToHost(q)
    Q.destroyQureg(q)
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec]
    if prec == 128:
        assert abs(tr - ref.total_prob()) <= PROB_TOL
        assert abs(pur - ref.purity()) <= PROB_TOL
        for t in range(N):
            assert abs(probs[t] - ref.prob_outcome(t, 1)) <= PROB_TOL
    else:
        d = 1 << N
        diag = got[np.arange(d) * (d + 1)].real
        assert abs(tr - float(np.sum(diag.astype(np.float64)))) <= PROB_TOL
        assert abs(pur - fsum_abs2(got)) <= PROB_TOL
        assert abs(tr - 1) <= 1e-5


# --------------------------------------------------------------- reductions
@pytest.mark.parametrize("prec", [128, 64])
def test_collapse_state_vector(Q, env, prec):
    n = 10
    ops = C.random_circuit(n, 8, 77, extras=True)
    for qubit, outcome in [(0, 0), (4, 1), (9, 1)]:
        ref = O.run_circuit(n, ops)
        pref = ref.collapse(qubit, outcome)
        Q.setEnvOption(env, "fusion", 1)
        q = Q.createQureg(n, prec, env)
        Q.applyCircuit(q, ops)
        p = Q.collapseToOutcome(q, qubit, outcome)
        got = Q.copyStateToHost(q)
        tot = Q.calcTotalProb(q)
        Q.destroyQureg(q)
        assert abs(p - pref) <= (PROB_TOL if prec == 128 else 1e-5)
        assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec]
        assert abs(tot - 1) <= (1e-13 if prec == 128 else 1e-5)


def general_gates(n, seed):
    """CNOT, controlled and plain general unitaries and phase shifts mixed
    into a random circuit (the layering itself has only H, sqrt(X), sqrt(Y),
    T, CZ, compactUnitary and multi-controlled phase flips)."""
    rng = C.SplitMix64(seed)
    ops = list(C.random_circuit(n, 6, seed, extras=n >= 3))
    for _ in range(3 * n):
        qs = C.distinct_qubits(rng, n, min(n, 3))
        a = C.haar_alpha_beta(rng)
        al, be = complex(a[0], a[1]), complex(a[2], a[3])
        u = (al.real, al.imag, -be.real, be.imag, be.real, be.imag, al.real, -al.imag)
        kind = rng.below(4)
        at = rng.below(len(ops) + 1)
        if kind == 0 and n >= 2:
            op = C.Op("CNOT", (qs[0],), (qs[1],))
        elif kind == 1 and n >= 2:
            op = C.Op("CUNITARY", (qs[0],), tuple(qs[1:]), u)
        elif kind == 2:
            op = C.Op("PHASE", (qs[0],), (), (0.3 + rng.uniform(),))
        else:
            op = C.Op("UNITARY", (qs[0],), (), u)
        ops.insert(at, op)
    return ops


@pytest.mark.parametrize("prec,arith", [(128, 0), (128, 1), (64, 0)])
@pytest.mark.parametrize("fusion", [0, 1])
@pytest.mark.parametrize("N", [3, 5])
def test_density_circuit_general_gates(Q, env, prec, arith, fusion, N):
    ops = C.with_noise(general_gates(N, 70 + N), 0.02, 0.01)
    ref = O.run_circuit(N, ops, density=True)
    Q.setEnvOption(env, "fusion", fusion)
    Q.setEnvOption(env, "arith", arith)
    try:
        q = Q.createDensityQureg(N, prec, env)
        Q.applyCircuit(q, ops)
        tr = Q.calcTotalProb(q)
        got = Q.copyStateToHost(q)
        Q.destroyQureg(q)
    finally:
        Q.setEnvOption(env, "arith", 0)
        Q.setEnvOption(env, "fusion", 1)
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec]
    assert abs(tr - ref.total_prob()) <= (PROB_TOL if prec == 128 else 1e-5)


@pytest.mark.parametrize("prec,arith", [(128, 0), (128, 1), (64, 0)])
@pytest.mark.parametrize("p_depol", [0.3, 0.75])
@pytest.mark.parametrize("N", [6, 7])
def test_density_circuit_heavy_noise(Q, env, prec, arith, p_depol, N):
    """Strong channels after every gate: the fused plan defers each qubit's
    off-diagonal factor (applied as a register-pair dephasing before the next
    pair update on the qubit), applies the common factor 1 - 2p/3 of each
    depolarising channel mid-plan once it passes 2^-30 (in order: over
    several passes a scale moved ahead of the growth it balances took
    double-float amplitudes below 2^-74 at a pass boundary), pairs a T's row
    and column phases into one off-diagonal op, and at p = 3/4 zeroes every
    off-diagonal entry of the qubit.  Against the unfused path and the
    oracle, with the trace and purity."""
    ops = C.with_noise(general_gates(N, 90), 0.3, p_depol)
    ref = O.run_circuit(N, ops, density=True)
    Q.setEnvOption(env, "arith", arith)
    try:
        got = {}
        for fusion in (1, 0):
            Q.setEnvOption(env, "fusion", fusion)
            q = Q.createDensityQureg(N, prec, env)
            Q.applyCircuit(q, ops)
            tr, pur = Q.calcTotalProb(q), Q.calcPurity(q)
            got[fusion] = Q.copyStateToHost(q)
            Q.destroyQureg(q)
            assert abs(tr - ref.total_prob()) <= (PROB_TOL if prec == 128 else 1e-5)
            assert abs(pur - ref.purity()) <= (1e-12 if prec == 128 else 1e-5)
    finally:
        Q.setEnvOption(env, "arith", 0)
        Q.setEnvOption(env, "fusion", 1)
    for fusion in (1, 0):
        assert np.max(np.abs(got[fusion] - ref.a)) <= AMP_TOL[prec], fusion


@pytest.mark.parametrize("prec,arith", [(128, 0), (128, 1), (64, 0)])
@pytest.mark.parametrize("n", [6, 11, 14])
def test_state_vector_general_gates(Q, env, prec, arith, n):
    ops = general_gates(n, 30 + n)
    ref = O.run_circuit(n, ops)
    Q.setEnvOption(env, "arith", arith)
    try:
        q = Q.createQureg(n, prec, env)
        Q.applyCircuit(q, ops)
        got = Q.copyStateToHost(q)
        Q.destroyQureg(q)
    finally:
        Q.setEnvOption(env, "arith", 0)
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec]


@pytest.mark.parametrize("prec", [128, 64])
def test_collapse_density(Q, env, prec):
    N = 4
    ops = C.random_density_circuit(N, 6, 8, 0.01, 0.005)
    ref = O.run_circuit(N, ops, density=True)
    pref = ref.collapse(2, 1)
    q = Q.createDensityQureg(N, prec, env)
    Q.applyCircuit(q, ops)
    p = Q.collapseToOutcome(q, 2, 1)
    got = Q.copyStateToHost(q)
    Q.destroyQureg(q)
    assert abs(p - pref) <= (PROB_TOL if prec == 128 else 1e-5)
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec]


def test_uniform_state_closed_forms(Q, env):
    n = 16
    q = Q.createQureg(n, 128, env)
    Q.initPlusState(q)
    for t in (0, 7, 15):
        assert abs(Q.calcProbOfOutcome(q, t, 0) - 0.5) <= PROB_TOL
    p = Q.collapseToOutcome(q, 5, 1)
    a = Q.copyStateToHost(q)
    Q.destroyQureg(q)
    assert abs(p - 0.5) <= PROB_TOL
    kept = ((np.arange(1 << n) >> 5) & 1) == 1
    assert np.max(np.abs(a[kept] - np.sqrt(2) * 2 ** (-n / 2))) <= 1e-15
    assert np.all(a[~kept] == 0)


# ------------------------------------------------------------ edge cases
def test_amplitude_ranges_and_ragged_copies(Q, env):
    n = 13
    psi = rand_state(n, 4)
    q = Q.createQureg(n, 128, env)
    Q.setAmps(q, psi[:1000], 0)
    Q.setAmps(q, psi[1000:], 1000)
    assert np.array_equal(Q.copyStateToHost(q), psi)
    assert np.array_equal(Q.copyStateToHost(q, 4095, 17), psi[4095:4112])
    assert Q.copyStateToHost(q, 5, 0).size == 0
    Q.destroyQureg(q)
    q = Q.createQureg(n, 64, env)
    Q.setAmps(q, psi)
    got = Q.copyStateToHost(q)
    assert np.max(np.abs(got - psi)) <= 1e-7
    Q.destroyQureg(q)


def test_errors_leave_state_unchanged(Q, env):
    n = 6
    psi = rand_state(n, 8)
    q = Q.createQureg(n, 128, env)
    Q.setAmps(q, psi)
    bad = [
        (lambda: Q.hadamard(q, n), "QS_E_QUBIT"),
        (lambda: Q.hadamard(q, -1), "QS_E_QUBIT"),
        (lambda: Q.controlledNot(q, 2, 2), "QS_E_DUP"),
        (lambda: Q.multiControlledPhaseFlip(q, [1, 3, 1]), "QS_E_DUP"),
        (lambda: Q.unitary(q, 0, [[1, 1], [0, 1]]), "QS_E_UNITARY"),
        (lambda: Q.compactUnitary(q, 0, 0.5, 0.5), "QS_E_UNITARY"),
        (lambda: Q.mixDephasing(q, 0, 0.1), "QS_E_NOT_DENSITY"),
        (lambda: Q.calcPurity(q), "QS_E_NOT_DENSITY"),
        (lambda: Q.calcProbOfOutcome(q, 0, 2), "QS_E_PROB"),
        (lambda: Q.applyCircuit(q, [C.Op("H", (0,)), C.Op("H", (9,))]), "QS_E_QUBIT"),
        (lambda: Q.copyStateToHost(q, 60, 10), "QS_E_ARG"),
    ]
    for f, name in bad:
        with pytest.raises(Q.QSimError) as e:
            f()
        assert e.value.name == name
    assert np.array_equal(Q.copyStateToHost(q), psi)
    Q.destroyQureg(q)
    with pytest.raises(Q.QSimError) as e:
        Q.hadamard(q, 0)
    assert e.value.name == "QS_E_HANDLE"
    d = Q.createDensityQureg(2, 128, env)
    for f in (lambda: Q.mixDephasing(d, 0, 0.51), lambda: Q.mixDepolarising(d, 1, 0.76)):
        with pytest.raises(Q.QSimError) as e:
            f()
        assert e.value.name == "QS_E_PROB"
    Q.destroyQureg(d)


def test_zero_probability_collapse_is_refused(Q, env):
    q = Q.createQureg(5, 128, env)
    with pytest.raises(Q.QSimError) as e:
        Q.collapseToOutcome(q, 3, 1)
    assert e.value.name == "QS_E_ZERO_PROB"
    a = Q.copyStateToHost(q)
    assert a[0] == 1 and np.all(a[1:] == 0)
    Q.destroyQureg(q)


def test_budget_and_torch_allocator(Q):
    import torch
    e = Q.createQuESTEnv()
    Q.setEnvOption(e, "budget_bytes", 1 << 20)
    with pytest.raises(Q.QSimError) as err:
        Q.createQureg(17, 128, e)          # 2 MiB > 1 MiB
    assert err.value.name == "QS_E_NOMEM"
    Q.setEnvOption(e, "budget_bytes", 0)
    Q.use_torch_allocator(e)
    before = torch.cuda.memory_allocated()
    q = Q.createQureg(20, 128, e)
    assert torch.cuda.memory_allocated() - before >= 16 << 20
    Q.hadamard(q, 3)
    assert abs(Q.calcProbOfOutcome(q, 3, 1) - 0.5) <= PROB_TOL
    s = torch.cuda.Stream()
    Q.setStream(e, s)
    Q.hadamard(q, 3)
    assert abs(Q.calcProbOfOutcome(q, 3, 0) - 1.0) <= PROB_TOL
    Q.destroyQureg(q)
    Q.destroyQuESTEnv(e)


# ------------------------------------------------ double-float arithmetic
@pytest.fixture
def df_env(Q, env):
    Q.setEnvOption(env, "arith", 1)
    yield env
    Q.setEnvOption(env, "arith", 0)


def test_double_float_every_gate(Q, df_env):
    n = 10
    psi = rand_state(n, 12)
    for op in single_ops(n, seed=5):
        ref = O.State(n, amps=psi)
        ref.apply(op)
        got = gpu_state(Q, df_env, n, [op], 128, fusion=1, init=psi)
        assert np.max(np.abs(got - ref.a)) <= 1e-13, op


@pytest.mark.parametrize("n", [9, 12, 16, 21])
def test_double_float_random_circuits(Q, df_env, n):
    ops = C.random_circuit(n, 24, 300 + n, extras=True)
    ref = O.run_circuit(n, ops)
    got = gpu_state(Q, df_env, n, ops, 128, fusion=1)
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[128]


@pytest.mark.parametrize("N", [5, 7])
def test_double_float_noisy_density(Q, df_env, N):
    ops = C.random_density_circuit(N, 10, 40 + N, 0.01, 0.005)
    ref = O.run_circuit(N, ops, density=True)
    q = Q.createDensityQureg(N, 128, df_env)
    Q.applyCircuit(q, ops)
    tr, pur = Q.calcTotalProb(q), Q.calcPurity(q)
    got = Q.copyStateToHost(q)
    Q.destroyQureg(q)
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[128]
    assert abs(tr - ref.total_prob()) <= PROB_TOL
    assert abs(pur - ref.purity()) <= PROB_TOL


def test_double_float_tiny_and_large_magnitudes(Q, df_env):
    """Amplitudes spanning many binades (down to 1e-30) convert and update
    within the absolute tolerance."""
    n = 10
    rng = np.random.default_rng(3)
    mags = 10.0 ** rng.uniform(-30, 0, size=1 << n)
    psi = mags * np.exp(1j * rng.uniform(0, 2 * np.pi, size=1 << n))
    psi /= np.linalg.norm(psi)
    ops = C.random_circuit(n, 6, 9, extras=True)
    ref = O.State(n, amps=psi).run(ops)
    got = gpu_state(Q, df_env, n, ops, 128, fusion=1, init=psi)
    assert np.max(np.abs(got - ref.a)) <= 1e-13


# ------------------------------------------------------- fused-pass counts
def test_fusion_cuts_passes_per_layer(Q, env):
    """A depth-40 layer has ~31 gates; fused tiles need far fewer HBM passes."""
    n = 24
    ops = C.random_circuit(n, 40, 8032, extras=True)
    Q.setEnvOption(env, "fusion", 1)
    q = Q.createQureg(n, 64, env)
    p0 = Q.getEnvOption(env, "fused_passes")
    Q.applyCircuit(q, ops)
    Q.syncQuESTEnv(env)
    passes = Q.getEnvOption(env, "fused_passes") - p0
    Q.destroyQureg(q)
    assert len(ops) / passes >= 4.0, (len(ops), passes)


def test_plan_cache_reuses_identical_gate_lists(Q, env):
    """A repeated flush of the same gate list reuses the cached plan (bit-
    identical result); a list differing in one angle is planned anew and
    matches the oracle."""
    n = 14
    ops = C.random_circuit(n, 10, 4242, extras=True)
    a = gpu_state(Q, env, n, ops, 128)
    h1 = Q.getEnvOption(env, "plan_cache_hits")
    b = gpu_state(Q, env, n, ops, 128)
    h2 = Q.getEnvOption(env, "plan_cache_hits")
    assert h2 > h1 and np.array_equal(a, b)
    i = next(j for j, o in enumerate(ops) if o.kind == "COMPACT")
    ar, ai, br, bi = ops[i].params
    c, s = np.cos(0.1), np.sin(0.1)
    ops2 = list(ops)
    ops2[i] = C.Op("COMPACT", ops[i].targets, (), (ar * c - ai * s, ar * s + ai * c, br, bi))
    got = gpu_state(Q, env, n, ops2, 128)
    assert Q.getEnvOption(env, "plan_cache_hits") == h2
    assert np.max(np.abs(got - O.run_circuit(n, ops2).a)) <= AMP_TOL[128]
