"""Multi-target (dense 2^m x 2^m) gates on the GPU against the CPU oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1802_08032_b300 import circuits as C
from gpu_helpers import AMP_TOL, gpu_state, rand_density_vec, rand_state

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


def rand_u(d, seed):
    rng = np.random.default_rng(seed)
    z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def cases(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for m in range(1, 6):
        for nc in (0, 1, 2):
            if m + nc > n:
                continue
            qs = [int(x) for x in rng.permutation(n)[:m + nc]]
            out.append((tuple(qs[:m]), tuple(qs[m:]), rand_u(1 << m, seed + 10 * m + nc)))
    return out


@pytest.mark.parametrize("prec,arith", [(128, 0), (128, 1), (64, 0)])
@pytest.mark.parametrize("fusion", [0, 1])
def test_multi_target_state_vector(Q, env, prec, arith, fusion):
    """arith 1: complex128 multi-target passes in double-float arithmetic."""
    n = 10
    psi = rand_state(n, 3)
    Q.setEnvOption(env, "fusion", fusion)
    Q.setEnvOption(env, "arith", arith)
    try:
        for targets, ctrls, U in cases(n, 100 + prec):
            ref = O.State(n, amps=psi)
            ref.multi(targets, U, ctrls)
            q = Q.createQureg(n, prec, env)
            Q.setAmps(q, psi)
            Q.multiControlledMultiQubitUnitary(q, ctrls, targets, U)
            got = Q.copyStateToHost(q)
            Q.destroyQureg(q)
            assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec] * (1 if prec == 128 else 0.1), \
                (targets, ctrls)
    finally:
        Q.setEnvOption(env, "arith", 0)
        Q.setEnvOption(env, "fusion", 1)


@pytest.mark.parametrize("prec,arith", [(128, 0), (128, 1), (64, 0)])
def test_multi_target_density_matrix(Q, env, prec, arith):
    N = 4
    rho = rand_density_vec(N, 6)
    Q.setEnvOption(env, "arith", arith)
    try:
        for targets, ctrls, U in cases(N, 7)[:8]:
            ref = O.State(N, density=True, amps=rho)
            ref.multi(targets, U, ctrls)
            d = Q.createDensityQureg(N, prec, env)
            Q.setAmps(d, rho)
            Q.multiControlledMultiQubitUnitary(d, ctrls, targets, U)
            got = Q.copyStateToHost(d)
            Q.destroyQureg(d)
            assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec] * (1 if prec == 128 else 0.1)
    finally:
        Q.setEnvOption(env, "arith", 0)


@pytest.mark.parametrize("prec", [128, 64])
def test_multi_between_fused_segments(Q, env, prec):
    """Fused single-target gates before, between and after multi-target gates."""
    n = 12
    ops = C.random_circuit(n, 8, 5, extras=True)
    U2, U3 = rand_u(4, 1), rand_u(8, 2)
    ref = O.State(n)
    Q.setEnvOption(env, "fusion", 1)
    q = Q.createQureg(n, prec, env)
    for i, chunk in enumerate((ops[:40], ops[40:90], ops[90:])):
        ref.run(chunk)
        Q.applyCircuit(q, chunk)
        if i == 0:
            ref.multi((3, 9), U2)
            Q.twoQubitUnitary(q, 3, 9, U2)
        elif i == 1:
            ref.multi((11, 0, 6), U3, (4,))
            Q.multiControlledMultiQubitUnitary(q, (4,), (11, 0, 6), U3)
    got = Q.copyStateToHost(q)
    Q.destroyQureg(q)
    assert np.max(np.abs(got - ref.a)) <= AMP_TOL[prec]


def test_multi_target_errors(Q, env):
    q = Q.createQureg(6, 128, env)
    psi = Q.copyStateToHost(q)
    bad = [
        (lambda: Q.multiQubitUnitary(q, (1, 1), np.eye(4)), "QS_E_DUP"),
        (lambda: Q.multiControlledMultiQubitUnitary(q, (2,), (2, 3), np.eye(4)), "QS_E_DUP"),
        (lambda: Q.multiQubitUnitary(q, (0, 1), 2 * np.eye(4)), "QS_E_UNITARY"),
        (lambda: Q.multiQubitUnitary(q, (0, 7), np.eye(4)), "QS_E_QUBIT"),
        (lambda: Q.multiQubitUnitary(q, tuple(range(6)), np.eye(64)), "QS_E_ARG"),
    ]
    for f, name in bad:
        with pytest.raises(Q.QSimError) as e:
            f()
        assert e.value.name == name
    assert np.array_equal(Q.copyStateToHost(q), psi)
    a = Q.createQureg(10, 64, env)
    Q.multiQubitUnitary(a, (0, 1), np.eye(4))
    with pytest.raises(Q.QSimError) as e:
        Q.createBatch(env, [a])
    assert e.value.name == "QS_E_ARG"
    Q.destroyQureg(a)
    Q.destroyQureg(q)


@pytest.mark.parametrize("m", [4, 5])
@pytest.mark.parametrize("ctrls", [(), (5, 17)])
@pytest.mark.parametrize("tset", [(0, 19, 7, 1, 12), (0, 1, 2, 3, 4), (9, 10, 11, 12, 13)])
def test_multi_target_tensor_cores(Q, env, m, ctrls, tset):
    """Complex64 gates on 4-5 targets on the tensor cores (three TF32
    products per FP32 operand pair; forced, and chosen by shape): many
    128-block tiles per CTA, targets mixed low and high, all among the
    lowest qubits or all above them, with and without controls; the staged
    kernel (every store form: straight from registers, through the stage
    in pairs or in single elements) and the register-gather kernel, against
    each other, the CUDA-core kernel and the oracle."""
    n = 20
    psi = rand_state(n, 40 + m)
    targets = tset[:m]
    U = rand_u(1 << m, 50 + m)
    ref = O.State(n, amps=psi)
    ref.multi(targets, U, ctrls)
    out = {}
    try:
        for tc, stage in ((2, 1), (1, 1), (2, 0), (0, 1)):
            Q.setEnvOption(env, "multi_tc", tc)
            Q.setEnvOption(env, "multi_tc_stage", stage)
            q = Q.createQureg(n, 64, env)
            Q.setAmps(q, psi)
            Q.multiControlledMultiQubitUnitary(q, ctrls, targets, U)
            Q.multiControlledMultiQubitUnitary(q, ctrls, targets, U.conj().T)
            Q.multiControlledMultiQubitUnitary(q, ctrls, targets, U)
            out[(tc, stage)] = Q.copyStateToHost(q)
            Q.destroyQureg(q)
    finally:
        Q.setEnvOption(env, "multi_tc", 1)
        Q.setEnvOption(env, "multi_tc_stage", 1)
    # three gates of 2^(m+1)-term FP32 sums whose products carry about 2^-23
    # relative error each (the TF32 split): bound 5e-6 of the largest
    # amplitude, well inside the complex64 bar of 1e-5 absolute
    scale = np.max(np.abs(ref.a))
    for key in ((2, 1), (1, 1), (2, 0)):
        assert np.max(np.abs(out[key] - ref.a)) <= 5e-6 * scale, key
        assert np.max(np.abs(out[key] - out[(0, 1)])) <= 5e-6 * scale, key
    # staged tiles (A in tensor memory) and register gathers (A in shared
    # memory) feed the same TF32 operands to the same products
    assert np.max(np.abs(out[(2, 1)] - out[(2, 0)])) <= 1e-6 * scale


@pytest.mark.parametrize("n", [10, 11, 12, 13])
def test_multi_target_tensor_cores_small_registers(Q, env, n):
    """Five targets on 10-13 qubits on the tensor cores: fewer than seven
    free qubits (one partial 128-block tile, the register-gather kernel) up
    to one and two full staged tiles, with the lowest target at qubit 0 and
    a control on qubit 0."""
    psi = rand_state(n, 80 + n)
    U = rand_u(32, 90 + n)
    Q.setEnvOption(env, "multi_tc", 2)
    try:
        for targets, ctrls in (((0, 3, n - 1, 5, 2), ()), ((4, 1, 6, 2, 7), (0,))):
            if n - len(targets) - len(ctrls) < 1:
                continue
            ref = O.State(n, amps=psi)
            ref.multi(targets, U, ctrls)
            q = Q.createQureg(n, 64, env)
            Q.setAmps(q, psi)
            Q.multiControlledMultiQubitUnitary(q, ctrls, targets, U)
            got = Q.copyStateToHost(q)
            Q.destroyQureg(q)
            assert np.max(np.abs(got - ref.a)) <= 5e-6 * np.max(np.abs(ref.a)), (targets, ctrls)
    finally:
        Q.setEnvOption(env, "multi_tc", 1)


def test_multi_target_tensor_cores_density_matrix(Q, env):
    N = 8
    rho = rand_density_vec(N, 9)
    U = rand_u(32, 77)
    ref = O.State(N, density=True, amps=rho)
    ref.multi((6, 0, 3, 7, 2), U, (5,))
    d = Q.createDensityQureg(N, 64, env)
    Q.setAmps(d, rho)
    Q.multiControlledMultiQubitUnitary(d, (5,), (6, 0, 3, 7, 2), U)
    got = Q.copyStateToHost(d)
    tr = Q.calcTotalProb(d)
    Q.destroyQureg(d)
    assert np.max(np.abs(got - ref.a)) <= 5e-6 * np.max(np.abs(ref.a))
    assert abs(tr - 1.0) <= 1e-5


def test_bounded_wait_reports_timeout(Q, env):
    """The tensor-core pass's bounded mbarrier wait, run on a barrier nothing
    arrives on: it gives up, the status word turns the next synchronisation
    into QS_E_TIMEOUT once, and the context stays usable."""
    Q.qsDiagBoundedWait(env, 2000)  # 2 ms
    with pytest.raises(Q.QSimError) as e:
        Q.syncQuESTEnv(env)
    assert e.value.name == "QS_E_TIMEOUT"
    Q.syncQuESTEnv(env)  # cleared
    Q.qsDiagBoundedWait(env, 500)
    q = Q.createQureg(6, 64, env)
    Q.hadamard(q, 0)
    with pytest.raises(Q.QSimError) as e:
        Q.calcTotalProb(q)  # a reduction reports it too
    assert e.value.name == "QS_E_TIMEOUT"
    assert abs(Q.calcTotalProb(q) - 1.0) < 1e-6
    Q.destroyQureg(q)
    with pytest.raises(Q.QSimError) as e:
        Q.qsDiagBoundedWait(env, 0)
    assert e.value.name == "QS_E_ARG"


_FACTOR_A = {}


def remap(ops, phys):
    """A gate list on qubits 0..len(phys)-1 moved onto the physical qubits phys."""
    return [C.Op(o.kind, tuple(phys[t] for t in o.targets), tuple(phys[c] for c in o.controls), o.params)
            for o in ops]


def gather_bits(idx, phys):
    """The bits of idx at the positions phys, packed in order (bit k = idx bit phys[k])."""
    out = np.zeros(len(idx), dtype=np.int64)
    for k, p in enumerate(phys):
        out |= ((idx >> p) & 1) << k
    return out


@pytest.mark.parametrize("prec,arith", [(128, 0), (128, 1), (64, 0)])
@pytest.mark.parametrize("m,targets,ctrls", [
    (5, (0, 19, 7, 1, 12), (5, 17)),   # targets mixed low and high, two controls
    (5, (0, 1, 2, 3, 4), (9,)),         # all among the lowest qubits
    (5, (25, 26, 27, 28, 29), ()),      # all at the top
    (4, (25, 26, 27, 28), (3,)),        # complex64: the paired-FMA CUDA-core pass
    (4, (1, 0, 3, 2), ()),              # complex64: shared-memory tiles in address order
    (3, (2, 0, 4), (1,)),               # the same with a control among the lowest qubits
])
def test_multi_target_30_qubits(Q, env, prec, arith, m, targets, ctrls):
    """A dense gate on a 30-qubit register (16 GiB complex128, 8 GiB
    complex64: 2^25 or more blocks, 64-bit indices) prepared as a product
    state: a seeded circuit on the 23-25 qubits A outside the gate, and one
    on the qubits B of the gate's targets and controls, then the gate.  The
    result is still a product, so each sampled amplitude is the oracle's
    factor-A amplitude times its factor-B amplitude (each factor run on its
    own, 2^25 amplitudes at most)."""
    n = 30
    B = sorted(set(targets) | set(ctrls))
    A = [q for q in range(n) if q not in B]
    loc = {p: k for k, p in enumerate(B)}
    U = rand_u(1 << m, 300 + m)
    ops_a = C.random_circuit(len(A), 4, 3000 + len(A), extras=True)
    ops_b = C.random_circuit(len(B), 6, 3100 + len(B), extras=True)
    key = tuple(A)
    if key not in _FACTOR_A:
        _FACTOR_A[key] = O.run_circuit(len(A), ops_a).a.copy()
    fa = _FACTOR_A[key]
    sb = O.run_circuit(len(B), ops_b)
    sb.multi(tuple(loc[t] for t in targets), U, tuple(loc[c] for c in ctrls))
    q = Q.createQureg(n, prec, env)
    Q.setEnvOption(env, "arith", arith)
    try:
        Q.applyCircuit(q, remap(ops_a, A) + remap(ops_b, B))
        Q.multiControlledMultiQubitUnitary(q, ctrls, targets, U)
        idx = np.array(C.sample_indices(n, 2048, 77 + m), dtype=np.int64)
        got = np.array([Q.copyStateToHost(q, int(i), 1)[0] for i in idx])
        tot = Q.calcTotalProb(q)
    finally:
        Q.setEnvOption(env, "arith", 0)
        Q.destroyQureg(q)
    want = fa[gather_bits(idx, A)] * sb.a[gather_bits(idx, B)]
    scale = np.max(np.abs(want))
    if prec == 128:
        assert np.max(np.abs(got - want)) <= AMP_TOL[128]
        assert np.max(np.abs(got - want)) <= 1e-10 * scale
        assert abs(tot - 1.0) <= 1e-12
    else:
        # the complex64 bar of 1e-5, taken relative to the largest sampled
        # amplitude (30-qubit amplitudes are ~1e-4, far below the absolute bar)
        assert np.max(np.abs(got - want)) <= 1e-5 * scale
        assert abs(tot - 1.0) <= 1e-5


@pytest.mark.parametrize("prec", [128, 64])
@pytest.mark.parametrize("m,targets,ctrls", [
    (5, (0, 9, 3, 1, 12), (5,)),   # targets mixed low and high in the row bits, one control
    (4, (10, 11, 12, 13), ()),     # the top row bits (their columns are the top vector bits)
])
def test_multi_target_density_matrix_14_qubits(Q, env, prec, m, targets, ctrls):
    """A dense gate on a noisy 14-qubit density matrix (2^28 amplitudes: 4 GiB
    complex128) prepared as a product rho_A (x) rho_B: a seeded noisy circuit
    on the qubits A outside the gate, one on the gate's qubits B, then the
    gate (U on the row bits, conj(U) on the column bits, Eq. 2).  Element
    (row, column) is rho_A(row_A, column_A) rho_B(row_B, column_B), each factor
    run by the oracle on its own."""
    N = 14
    B = sorted(set(targets) | set(ctrls))
    A = [q for q in range(N) if q not in B]
    loc = {p: k for k, p in enumerate(B)}
    U = rand_u(1 << m, 400 + m)
    ops_a = C.with_noise(C.random_circuit(len(A), 4, 1400 + len(A), extras=True), 0.01, 0.005)
    ops_b = C.with_noise(C.random_circuit(len(B), 6, 1500 + len(B), extras=True), 0.01, 0.005)
    sa = O.run_circuit(len(A), ops_a, density=True)
    sb = O.run_circuit(len(B), ops_b, density=True)
    sb.multi(tuple(loc[t] for t in targets), U, tuple(loc[c] for c in ctrls))
    d = Q.createDensityQureg(N, prec, env)
    try:
        Q.applyCircuit(d, remap(ops_a, A) + remap(ops_b, B))
        Q.multiControlledMultiQubitUnitary(d, ctrls, targets, U)
        idx = np.array(C.sample_indices(2 * N, 2048, 91 + m), dtype=np.int64)
        got = np.array([Q.copyStateToHost(d, int(i), 1)[0] for i in idx])
        tr = Q.calcTotalProb(d)
    finally:
        Q.destroyQureg(d)
    # vector index = row + 2^N column: factor X's element sits at its row bits
    # (positions X) and its column bits (positions X + N)
    ia = gather_bits(idx, A + [q + N for q in A])
    ib = gather_bits(idx, B + [q + N for q in B])
    want = sa.a[ia] * sb.a[ib]
    scale = np.max(np.abs(want))
    if prec == 128:
        assert np.max(np.abs(got - want)) <= AMP_TOL[128]
        assert np.max(np.abs(got - want)) <= 1e-10 * scale
        assert abs(tr - 1.0) <= 1e-12
    else:
        assert np.max(np.abs(got - want)) <= 1e-5 * scale
        assert abs(tr - 1.0) <= 1e-5


@pytest.mark.parametrize("mode,stage", [(0, 1), (1, 1), (2, 1), (2, 0)])
def test_multi_target_random_placements(Q, env, mode, stage):
    """Complex64 gates on 2-5 targets at seeded random positions, most with a
    target among the five lowest qubits and some with controls there too
    (every table the shared-memory tile and tensor-core paths derive from
    the positions), on 16 qubits, each against the oracle."""
    n = 16
    rng = np.random.default_rng(500 + mode)
    psi = rand_state(n, 61)
    Q.setEnvOption(env, "multi_tc", mode)
    Q.setEnvOption(env, "multi_tc_stage", stage)
    try:
        for case in range(24):
            m = int(rng.integers(2, 6))
            nc = int(rng.integers(0, 3))
            low = rng.permutation(6)[: int(rng.integers(1, min(m, 3) + 1))]
            rest = [q for q in rng.permutation(n) if q not in low]
            qs = [int(q) for q in low] + [int(q) for q in rest]
            targets, ctrls = tuple(qs[:m]), tuple(qs[m:m + nc])
            if case % 3 == 0 and nc > 0:  # a control among the lowest qubits
                ctrls = (targets[0],) + ctrls[1:]
                targets = (qs[m + nc],) + targets[1:]
            U = rand_u(1 << m, 700 + 31 * mode + case)
            ref = O.State(n, amps=psi)
            ref.multi(targets, U, ctrls)
            q = Q.createQureg(n, 64, env)
            Q.setAmps(q, psi)
            Q.multiControlledMultiQubitUnitary(q, ctrls, targets, U)
            got = Q.copyStateToHost(q)
            Q.destroyQureg(q)
            assert np.max(np.abs(got - ref.a)) <= 5e-6 * np.max(np.abs(ref.a)), (m, targets, ctrls)
    finally:
        Q.setEnvOption(env, "multi_tc", 1)
        Q.setEnvOption(env, "multi_tc_stage", 1)
