"""Pins of the CPU oracle against things other than itself (CPU only).

Dense 2^n x 2^n Kronecker matrices (Eq. 1 and its controlled form), the
textbook identity vec(U rho U^dagger) = (U* (x) U) vec(rho) behind Eq. 2,
brute-force Kraus sums, closed forms and invariants.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1802_08032_b300 import circuits as C

RNG = np.random.default_rng(20180222)


def rand_state(nq, rng=RNG):
    v = rng.normal(size=1 << nq) + 1j * rng.normal(size=1 << nq)
    return v / np.linalg.norm(v)


def rand_unitary(rng=RNG):
    z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def rand_density(N, rng=RNG):
    d = 1 << N
    A = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    rho = A @ A.conj().T
    return rho / np.trace(rho)


def vec(rho):
    """Column-stacked vectorisation: index j + 2^N k holds rho[j, k]."""
    return np.ascontiguousarray(rho.T.reshape(-1))


def kron_list(factors):
    """factors[q] acts on qubit q; qubit q is bit q of the index, so the
    Kronecker product runs from the highest qubit down."""
    out = np.ones((1, 1), dtype=np.complex128)
    for f in reversed(factors):
        out = np.kron(out, f)
    return out


def dense_controlled(n, t, ctrls, G):
    """I + (|1><1| on every control) (x) (G - I on the target)."""
    factors = [O.MAT_I] * n
    for c in ctrls:
        factors[c] = np.array([[0, 0], [0, 1]], dtype=np.complex128)
    factors[t] = G - O.MAT_I
    return np.eye(1 << n, dtype=np.complex128) + kron_list(factors)


GATES = ["H", "T", "SX", "SY", "X", "COMPACT", "UNITARY"]


def gate_for(kind):
    if kind == "COMPACT":
        g = C.haar_alpha_beta(C.SplitMix64(int(RNG.integers(1 << 62))))
        return O.compact_matrix(*g)
    if kind == "UNITARY":
        return rand_unitary()
    return O.gate_matrix(kind)


@pytest.mark.parametrize("kind", GATES)
def test_gate_matches_dense_kronecker(kind):
    n = 6
    for t in range(n):
        others = [q for q in range(n) if q != t]
        for nc in range(4):
            ctrls = tuple(int(c) for c in RNG.choice(others, size=nc, replace=False))
            G = gate_for(kind)
            psi = rand_state(n)
            s = O.State(n, amps=psi)
            s.gate(t, G, ctrls)
            ref = dense_controlled(n, t, ctrls, G) @ psi
            assert np.max(np.abs(s.a - ref)) < 1e-14, (kind, t, ctrls)


def test_named_matrices_are_textbook():
    # (sqrt X)^2 = X, (sqrt Y)^2 = Y, T^2 = S = diag(1, i), H^2 = I
    assert np.allclose(O.MAT_SX @ O.MAT_SX, O.MAT_X, atol=1e-15)
    assert np.allclose(O.MAT_SY @ O.MAT_SY, O.MAT_Y, atol=1e-15)
    assert np.allclose(O.MAT_T @ O.MAT_T, np.diag([1, 1j]), atol=1e-15)
    assert np.allclose(O.MAT_H @ O.MAT_H, np.eye(2), atol=1e-15)
    for M in (O.MAT_H, O.MAT_T, O.MAT_SX, O.MAT_SY):
        assert np.allclose(M @ M.conj().T, np.eye(2), atol=1e-15)
    a, b = 0.6 + 0.0j, 0.0 + 0.8j
    U = O.compact_matrix(a.real, a.imag, b.real, b.imag)
    assert np.allclose(U @ U.conj().T, np.eye(2), atol=1e-15)
    assert abs(np.linalg.det(U) - 1) < 1e-15          # SU(2) parameterisation
    assert U[0, 0] == a and U[1, 0] == b


def test_phase_flip_matches_dense_diagonal():
    n = 7
    for qs in [(0, 1), (2, 6), (1, 3, 5), (0, 2, 4, 6), (6,)]:
        psi = rand_state(n)
        s = O.State(n, amps=psi)
        s.phase_flip(qs)
        mask = sum(1 << q for q in qs)
        d = np.array([-1.0 if (j & mask) == mask else 1.0 for j in range(1 << n)])
        assert np.array_equal(s.a, d * psi)                 # exact sign pattern


def test_cnot_is_exact_permutation():
    n = 6
    for c, t in [(0, 1), (5, 0), (2, 4)]:
        psi = rand_state(n)
        s = O.State(n, amps=psi)
        s.apply(C.Op("CNOT", (t,), (c,)))
        perm = np.array([j ^ (1 << t) if (j >> c) & 1 else j for j in range(1 << n)])
        assert np.array_equal(s.a, psi[perm])


def test_hadamard_all_gives_uniform():
    for n in (1, 5, 10):
        s = O.State(n)
        for q in range(n):
            s.gate(q, O.MAT_H)
        assert np.max(np.abs(s.a - 2 ** (-n / 2))) < 1e-15


def test_gate_then_dagger_is_identity():
    n = 8
    psi = rand_state(n)
    s = O.State(n, amps=psi)
    gates = [(int(RNG.integers(n)), rand_unitary()) for _ in range(30)]
    for t, G in gates:
        s.gate(t, G)
    for t, G in reversed(gates):
        s.gate(t, G.conj().T)
    assert np.max(np.abs(s.a - psi)) < 1e-13


def test_norm_preserved_random_circuit():
    s = O.run_circuit(10, C.random_circuit(10, 30, 7, extras=True))
    assert abs(s.total_prob() - 1) < 1e-14


# ---------------------------------------------------------------- density
def dense_kraus(N, t, ops, rho):
    out = np.zeros_like(rho)
    for K in ops:
        f = [O.MAT_I] * N
        f[t] = K
        Kf = kron_list(f)
        out += Kf @ rho @ Kf.conj().T
    return out


def test_dm_gate_matches_u_rho_udagger():
    N = 3
    for t in range(N):
        for ctrls in [(), ((t + 1) % N,), tuple(q for q in range(N) if q != t)]:
            U = rand_unitary()
            rho = rand_density(N)
            s = O.State(N, density=True, amps=vec(rho))
            s.gate(t, U, ctrls)
            Uf = dense_controlled(N, t, ctrls, U)
            ref = Uf @ rho @ Uf.conj().T
            assert np.max(np.abs(s.matrix() - ref)) < 1e-14
            # the same via the superoperator (U* (x) U) on the column-stacked vector
            assert np.max(np.abs(s.a - np.kron(Uf.conj(), Uf) @ vec(rho))) < 1e-14


def test_dm_phase_flip_matches_dense():
    N = 3
    rho = rand_density(N)
    s = O.State(N, density=True, amps=vec(rho))
    s.phase_flip((0, 2))
    P = np.diag([-1.0 if (j & 5) == 5 else 1.0 for j in range(8)])
    assert np.max(np.abs(s.matrix() - P @ rho @ P)) < 1e-15


@pytest.mark.parametrize("channel", ["dephase", "depol"])
def test_kraus_channel_matches_dense(channel):
    N = 3
    for t in range(N):
        for p in (0.0, 0.01, 0.3):
            ops = O.kraus_dephasing(p) if channel == "dephase" else O.kraus_depolarising(p)
            rho = rand_density(N)
            s = O.State(N, density=True, amps=vec(rho))
            s.kraus(t, ops)
            assert np.max(np.abs(s.matrix() - dense_kraus(N, t, ops, rho))) < 1e-15


def test_dephasing_closed_form():
    N, t, p, m = 3, 1, 0.07, 5
    rho = rand_density(N)
    s = O.State(N, density=True, amps=vec(rho))
    for _ in range(m):
        s.apply(C.Op("DEPHASE", (t,), (), (p,)))
    d = 1 << N
    for j in range(d):
        for k in range(d):
            f = (1 - 2 * p) ** m if ((j >> t) & 1) != ((k >> t) & 1) else 1.0
            assert abs(s.matrix()[j, k] - f * rho[j, k]) < 1e-15


def test_depolarising_shrinks_bloch_vector():
    p = 0.2
    rho = rand_density(1)
    s = O.State(1, density=True, amps=vec(rho))
    s.apply(C.Op("DEPOL", (0,), (), (p,)))

    def bloch(r):
        return np.array([np.trace(r @ P).real for P in (O.MAT_X, O.MAT_Y, O.MAT_Z)])

    assert np.max(np.abs(bloch(s.matrix()) - (1 - 4 * p / 3) * bloch(rho))) < 1e-15
    s.apply(C.Op("DEPOL", (0,), (), (0.75,)))
    assert np.max(np.abs(s.matrix() - np.eye(2) / 2)) < 1e-15


def test_pure_circuit_density_equals_outer_product():
    N = 4
    ops = C.random_circuit(N, 8, 99, extras=True)
    sv = O.run_circuit(N, ops)
    dm = O.run_circuit(N, ops, density=True)
    assert np.max(np.abs(dm.matrix() - np.outer(sv.a, sv.a.conj()))) < 1e-14
    assert abs(dm.purity() - 1) < 1e-14


def test_noisy_circuit_trace_hermitian_purity():
    N = 4
    dm = O.run_circuit(N, C.random_density_circuit(N, 10, 3, 0.01, 0.005), density=True)
    R = dm.matrix()
    assert abs(dm.total_prob() - 1) < 1e-14
    assert np.max(np.abs(R - R.conj().T)) < 1e-15
    assert dm.purity() < 1 - 1e-3
    assert abs(dm.purity() - np.trace(R @ R).real) < 1e-14
    assert np.min(np.linalg.eigvalsh(R)) > -1e-14
    for q in range(N):
        assert abs(dm.prob_outcome(q, 0) + dm.prob_outcome(q, 1) - 1) < 1e-14


# ---------------------------------------------------------------- reductions
def test_reductions_closed_forms():
    n = 9
    s = O.State(n)
    for q in range(n):
        s.gate(q, O.MAT_H)
    for q in range(n):
        assert abs(s.prob_outcome(q, 0) - 0.5) < 1e-15
    b = O.State(n)                     # basis state |0...0> then X on qubit 3
    b.gate(3, O.MAT_X)
    assert b.prob_outcome(3, 1) == 1.0 and b.prob_outcome(3, 0) == 0.0
    assert b.prob_outcome(2, 0) == 1.0


def test_reduction_accuracy_vs_exact_sum():
    psi = rand_state(14) * 1.3
    s = O.State(14, amps=psi)
    exact = math.fsum((psi.real ** 2).tolist() + (psi.imag ** 2).tolist())
    assert abs(s.total_prob() - exact) <= 2e-16 * exact
    sel = [(j >> 5) & 1 == 1 for j in range(1 << 14)]
    exact1 = math.fsum((psi[sel].real ** 2).tolist() + (psi[sel].imag ** 2).tolist())
    assert abs(s.prob_outcome(5, 1) - exact1) <= 2e-16 * exact1


def test_collapse_sv():
    n = 8
    s = O.State(n)
    for q in range(n):
        s.gate(q, O.MAT_H)
    p = s.collapse(2, 1)
    assert abs(p - 0.5) < 1e-15
    kept = [(j >> 2) & 1 == 1 for j in range(1 << n)]
    assert np.max(np.abs(s.a[kept] - math.sqrt(2) * 2 ** (-n / 2))) < 1e-15
    assert np.all(s.a[[not k for k in kept]] == 0)
    assert abs(s.prob_outcome(2, 1) - 1) < 1e-15 and abs(s.total_prob() - 1) < 1e-15


def test_collapse_dm():
    N = 3
    rho = rand_density(N)
    s = O.State(N, density=True, amps=vec(rho))
    p = s.collapse(1, 0)
    P = np.diag([1.0 if ((j >> 1) & 1) == 0 else 0.0 for j in range(8)])
    ref = P @ rho @ P / np.trace(P @ rho).real
    assert abs(p - np.trace(P @ rho).real) < 1e-15
    assert np.max(np.abs(s.matrix() - ref)) < 1e-15
    assert abs(s.total_prob() - 1) < 1e-15 and abs(s.prob_outcome(1, 0) - 1) < 1e-15


# ---------------------------------------------------------------- multi-qubit
def rand_unitary_n(d, rng=RNG):
    z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def dense_multi(n, targets, U, ctrls=()):
    """Full matrix from the definition: <i|M|j> = U[sub(i), sub(j)] when i and
    j agree outside the targets and the controls of j are all 1, where sub
    collects the target bits (bit k = targets[k])."""
    dim = 1 << n
    tmask = sum(1 << t for t in targets)
    cmask = sum(1 << c for c in ctrls)
    sub = [sum(((i >> t) & 1) << k for k, t in enumerate(targets)) for i in range(dim)]
    M = np.zeros((dim, dim), dtype=np.complex128)
    for j in range(dim):
        if (j & cmask) != cmask:
            M[j, j] = 1
            continue
        for i in range(dim):
            if (i & ~tmask) == (j & ~tmask):
                M[i, j] = U[sub[i], sub[j]]
    return M


def test_multi_of_kronecker_product_equals_single_gates():
    n = 6
    A, B = rand_unitary(), rand_unitary()
    for t0, t1 in [(0, 1), (4, 2), (5, 0)]:
        psi = rand_state(n)
        s = O.State(n, amps=psi)
        s.multi((t0, t1), np.kron(B, A))          # bit 0 of U's index is t0
        r = O.State(n, amps=psi)
        r.gate(t0, A)
        r.gate(t1, B)
        assert np.max(np.abs(s.a - r.a)) < 1e-14


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_multi_matches_dense_definition(m):
    n = 6
    for trial in range(3):
        targets = tuple(int(x) for x in RNG.choice(n, size=m, replace=False))
        others = [q for q in range(n) if q not in targets]
        ctrls = tuple(int(x) for x in RNG.choice(others, size=min(trial, len(others)), replace=False))
        U = rand_unitary_n(1 << m)
        psi = rand_state(n)
        s = O.State(n, amps=psi)
        s.multi(targets, U, ctrls)
        assert np.max(np.abs(s.a - dense_multi(n, targets, U, ctrls) @ psi)) < 1e-14


def test_multi_permutation_is_exact():
    """The 2-qubit SWAP as a dense matrix is an exact permutation."""
    n = 5
    SWAP = np.eye(4, dtype=np.complex128)[[0, 2, 1, 3]]
    psi = rand_state(n)
    s = O.State(n, amps=psi)
    s.multi((1, 3), SWAP)
    perm = [(j & ~0b1010) | (((j >> 1) & 1) << 3) | (((j >> 3) & 1) << 1) for j in range(1 << n)]
    assert np.array_equal(s.a, psi[perm])


def test_dm_multi_matches_u_rho_udagger():
    N = 3
    for targets, ctrls in [((0, 2), ()), ((2, 1), (0,)), ((1,), (2,))]:
        U = rand_unitary_n(1 << len(targets))
        rho = rand_density(N)
        s = O.State(N, density=True, amps=vec(rho))
        s.multi(targets, U, ctrls)
        Uf = dense_multi(N, targets, U, ctrls)
        assert np.max(np.abs(s.matrix() - Uf @ rho @ Uf.conj().T)) < 1e-14
