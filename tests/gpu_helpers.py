"""Helpers shared by the GPU parity tests (no GPU needed to import)."""
import math

import numpy as np

from paper_1802_08032_b300 import circuits as C

# Parity bars: max |amplitude difference| after the circuit.
AMP_TOL = {128: 1e-12, 64: 1e-5}
PROB_TOL = 1e-13


def rand_state(nq, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=1 << nq) + 1j * rng.normal(size=1 << nq)
    return v / np.linalg.norm(v)


def rand_density_vec(N, seed):
    rng = np.random.default_rng(seed)
    d = 1 << N
    A = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    rho = A @ A.conj().T
    rho /= np.trace(rho).real
    return np.ascontiguousarray(rho.T.reshape(-1))


def rand_unitary_params(seed):
    rng = np.random.default_rng(seed)
    z = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    q, r = np.linalg.qr(z)
    u = q * (np.diag(r) / np.abs(np.diag(r)))
    return tuple(x for c in u.reshape(-1) for x in (c.real, c.imag))


def single_ops(n, seed=0):
    """One op of every kind on every target (with several control patterns)."""
    rng = C.SplitMix64(seed)
    ops = []
    for t in range(n):
        others = [q for q in range(n) if q != t]
        for k in ("H", "X", "SX", "SY", "T"):
            ops.append(C.Op(k, (t,)))
        ops.append(C.Op("PHASE", (t,), (), (0.3 + t,)))
        ops.append(C.Op("COMPACT", (t,), (), C.haar_alpha_beta(rng)))
        ops.append(C.Op("UNITARY", (t,), (), rand_unitary_params(seed * 1000 + t)))
        for nc in range(1, min(4, n)):
            ctr = tuple(others[(rng.below(len(others)) + i * 3) % len(others)] for i in range(nc))
            if len(set(ctr)) < nc:
                continue
            ops.append(C.Op("CUNITARY", (t,), ctr, rand_unitary_params(seed * 7 + t + nc)))
        if others:
            c = others[rng.below(len(others))]
            ops.append(C.Op("CNOT", (t,), (c,)))
            ops.append(C.Op("CZ", (min(t, c), max(t, c))))
        for nc in range(1, min(5, n + 1)):
            qs = C.distinct_qubits(rng, n, nc)
            ops.append(C.Op("MCPF", (), qs))
    return ops


def gpu_state(Q, env, n, ops, prec, density=False, fusion=1, init=None):
    Q.setEnvOption(env, "fusion", fusion)
    q = (Q.createDensityQureg if density else Q.createQureg)(n, prec, env)
    try:
        if init is not None:
            Q.setAmps(q, init)
        Q.applyCircuit(q, ops)
        return Q.copyStateToHost(q)
    finally:
        Q.destroyQureg(q)


def fsum_abs2(v):
    return math.fsum((v.real ** 2).tolist() + (v.imag ** 2).tolist())


def inverse(ops):
    """C-dagger of a gate list: the inverse of each gate, in reverse order.
    sqrt(X) and sqrt(Y) are principal square roots, (1/2)[[1+i, 1-i], [1-i, 1+i]]
    and ((1+i)/2)[[1, -1], [1, 1]]; their inverses are the conjugate
    transposes.  compactUnitary(a, b) = [[a, -b*], [b, a*]] has the inverse
    compactUnitary(a*, -b)."""
    sx_dag = (0.5, -0.5, 0.5, 0.5, 0.5, 0.5, 0.5, -0.5)
    sy_dag = (0.5, -0.5, 0.5, -0.5, -0.5, 0.5, 0.5, -0.5)
    out = []
    for o in reversed(ops):
        if o.kind in (C.H, C.CZ, C.MCPF):
            out.append(o)
        elif o.kind == C.T_GATE:
            out.append(C.Op(C.PHASE, o.targets, (), (-np.pi / 4,)))
        elif o.kind == C.SQRT_X:
            out.append(C.Op(C.UNITARY, o.targets, (), sx_dag))
        elif o.kind == C.SQRT_Y:
            out.append(C.Op(C.UNITARY, o.targets, (), sy_dag))
        elif o.kind == C.COMPACT:
            ar, ai, br, bi = o.params
            out.append(C.Op(C.COMPACT, o.targets, (), (ar, -ai, -br, -bi)))
        else:
            raise AssertionError(o.kind)
    return out
