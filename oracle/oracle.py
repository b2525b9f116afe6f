"""CPU oracle: plain FP64 simulation of gate lists (TEST INFRASTRUCTURE ONLY).

Only tests, the smoke check and the benchmark's CPU-baseline leg may import
this module.  It shares nothing with the CUDA library: the C core
(qsim_oracle.c) is compiled here with gcc, and the gate matrices below are
this module's own textbook definitions.  The only thing it has in common
with the CUDA path is its input: gate lists (kind, targets, controls,
params) as produced by the seeded generator.

Gate matrices (named in the paper's benchmark set, Sec. II.C; the paper
prints no matrices, these are the textbook ones):
  H = [[1, 1], [1, -1]] / sqrt(2)            T = diag(1, exp(i pi/4))
  sqrt(X) = [[1+i, 1-i], [1-i, 1+i]] / 2      sqrt(Y) = (1+i)/2 [[1, -1], [1, 1]]
  X = [[0, 1], [1, 0]]                        Z = diag(1, -1)
  phaseShift(phi) = diag(1, exp(i phi))
  compactUnitary(alpha, beta) = [[alpha, -conj(beta)], [beta, conj(alpha)]]
Noise channels (the paper names dephasing and depolarising noise, Sec. I
and II.B.1, without formulas; readings):
  dephasing(p):    Kraus {sqrt(1-p) I, sqrt(p) Z},                 p in [0, 1/2]
  depolarising(p): Kraus {sqrt(1-p) I, sqrt(p/3) X, sqrt(p/3) Y,
                          sqrt(p/3) Z},                            p in [0, 3/4]
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "qsim_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

SQ2 = np.sqrt(0.5)
MAT_H = np.array([[1, 1], [1, -1]], dtype=np.complex128) * SQ2
MAT_T = np.array([[1, 0], [0, np.exp(1j * np.pi / 4)]], dtype=np.complex128)
MAT_SX = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
MAT_SY = 0.5 * (1 + 1j) * np.array([[1, -1], [1, 1]], dtype=np.complex128)
MAT_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
MAT_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
MAT_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
MAT_I = np.eye(2, dtype=np.complex128)


def compact_matrix(ar, ai, br, bi):
    a, b = complex(ar, ai), complex(br, bi)
    return np.array([[a, -np.conj(b)], [b, np.conj(a)]], dtype=np.complex128)


def params_matrix(params):
    v = np.array(params, dtype=np.float64).reshape(4, 2)
    return (v[:, 0] + 1j * v[:, 1]).reshape(2, 2)


def kraus_dephasing(p):
    return [np.sqrt(1 - p) * MAT_I, np.sqrt(p) * MAT_Z]


def kraus_depolarising(p):
    s = np.sqrt(p / 3)
    return [np.sqrt(1 - p) * MAT_I, s * MAT_X, s * MAT_Y, s * MAT_Z]


_FIXED = {"H": MAT_H, "T": MAT_T, "SX": MAT_SX, "SY": MAT_SY, "X": MAT_X, "CNOT": MAT_X}


def gate_matrix(kind, params=()):
    if kind in _FIXED:
        return _FIXED[kind]
    if kind == "COMPACT":
        return compact_matrix(*params)
    if kind == "PHASE":
        return np.array([[1, 0], [0, np.exp(1j * params[0])]], dtype=np.complex128)
    if kind in ("UNITARY", "CUNITARY"):
        return params_matrix(params)
    raise ValueError(f"oracle: no matrix for {kind}")


# --------------------------------------------------------------------------
def build_library(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build_library())
        P, I, U64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
        sig = {
            "orc_init_zero": [P, I], "orc_init_plus": [P, I],
            "orc_apply_gate": [P, I, I, U64, P], "orc_phase_flip": [P, I, U64],
            "orc_apply_dm_gate": [P, I, I, U64, P], "orc_dm_phase_flip": [P, I, U64],
            "orc_apply_kraus": [P, I, I, I, P],
            "orc_total_prob_sv": [P, I], "orc_prob_outcome_sv": [P, I, I, I],
            "orc_total_prob_dm": [P, I], "orc_prob_outcome_dm": [P, I, I, I],
            "orc_purity_dm": [P, I],
            "orc_collapse_sv": [P, I, I, I, D], "orc_collapse_dm": [P, I, I, I, D],
            "orc_apply_multi": [P, I, P, I, U64, P], "orc_apply_dm_multi": [P, I, P, I, U64, P],
            "orc_num_threads": [], "orc_set_num_threads": [I],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = D if name.startswith(("orc_total", "orc_prob", "orc_purity")) else (
                I if name == "orc_num_threads" else None)
        _lib = L
    return _lib


def _ptr(a):
    assert a.dtype == np.complex128 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _cmat(m):
    return np.ascontiguousarray(np.asarray(m, dtype=np.complex128).reshape(-1))


def _mask(qs):
    m = 0
    for q in qs:
        m |= 1 << q
    return m


# --------------------------------------------------------------------------
class State:
    """An oracle register: n-qubit state vector, or N-qubit density matrix
    stored as the 2N-qubit vector of Eq. 2."""

    def __init__(self, n, density=False, amps=None):
        self.n = n
        self.density = density
        self.nq = 2 * n if density else n
        if amps is None:
            self.a = np.empty(1 << self.nq, dtype=np.complex128)
            lib().orc_init_zero(_ptr(self.a), self.nq)
        else:
            self.a = np.ascontiguousarray(amps, dtype=np.complex128).copy()
            assert self.a.size == 1 << self.nq

    # -- gates -------------------------------------------------------------
    def _check_qubits(self, qs):
        # the C core does no bounds checks: reject bad qubits here
        for q in qs:
            if not 0 <= int(q) < self.n:
                raise ValueError(f"oracle: qubit {q} outside an {self.n}-qubit register")
        if len(set(int(q) for q in qs)) != len(qs):
            raise ValueError(f"oracle: repeated qubit in {tuple(qs)}")

    def gate(self, q, g, controls=()):
        self._check_qubits((q,) + tuple(controls))
        g = _cmat(g)
        if self.density:
            lib().orc_apply_dm_gate(_ptr(self.a), self.n, q, _mask(controls), g.ctypes.data)
        else:
            lib().orc_apply_gate(_ptr(self.a), self.n, q, _mask(controls), g.ctypes.data)

    def phase_flip(self, qubits):
        self._check_qubits(tuple(qubits))
        if self.density:
            lib().orc_dm_phase_flip(_ptr(self.a), self.n, _mask(qubits))
        else:
            lib().orc_phase_flip(_ptr(self.a), self.n, _mask(qubits))

    def multi(self, targets, U, controls=()):
        """Dense 2^m x 2^m gate U on `targets` (bit k of U's index is
        targets[k]), restricted to the controls."""
        self._check_qubits(tuple(targets) + tuple(controls))
        m = len(targets)
        U = _cmat(U)
        assert U.size == 4 ** m and 1 <= m <= 6
        t = (ctypes.c_int * m)(*targets)
        if self.density:
            lib().orc_apply_dm_multi(_ptr(self.a), self.n, t, m, _mask(controls), U.ctypes.data)
        else:
            lib().orc_apply_multi(_ptr(self.a), self.n, t, m, _mask(controls), U.ctypes.data)

    def kraus(self, q, ops):
        assert self.density
        self._check_qubits((q,))
        K = _cmat(np.stack(ops))
        lib().orc_apply_kraus(_ptr(self.a), self.n, q, len(ops), K.ctypes.data)

    def apply(self, op):
        k = op.kind
        if k in ("H", "T", "SX", "SY", "X", "PHASE", "COMPACT", "UNITARY"):
            self.gate(op.targets[0], gate_matrix(k, op.params))
        elif k in ("CNOT", "CUNITARY"):
            self.gate(op.targets[0], gate_matrix(k, op.params), op.controls)
        elif k == "CZ":
            self.phase_flip(op.targets)
        elif k == "MCPF":
            self.phase_flip(op.controls)
        elif k == "DEPHASE":
            self.kraus(op.targets[0], kraus_dephasing(op.params[0]))
        elif k == "DEPOL":
            self.kraus(op.targets[0], kraus_depolarising(op.params[0]))
        elif k == "MULTI":
            m = len(op.targets)
            v = np.array(op.params, dtype=np.float64).reshape(-1, 2)
            self.multi(op.targets, (v[:, 0] + 1j * v[:, 1]).reshape(1 << m, 1 << m), op.controls)
        else:
            raise ValueError(f"oracle: unknown op {k}")

    def run(self, ops):
        for op in ops:
            self.apply(op)
        return self

    # -- reductions --------------------------------------------------------
    def total_prob(self):
        if self.density:
            return lib().orc_total_prob_dm(_ptr(self.a), self.n)
        return lib().orc_total_prob_sv(_ptr(self.a), self.n)

    def prob_outcome(self, q, outcome):
        self._check_qubits((q,))
        if self.density:
            return lib().orc_prob_outcome_dm(_ptr(self.a), self.n, q, outcome)
        return lib().orc_prob_outcome_sv(_ptr(self.a), self.n, q, outcome)

    def purity(self):
        assert self.density
        return lib().orc_purity_dm(_ptr(self.a), self.n)

    def collapse(self, q, outcome):
        p = self.prob_outcome(q, outcome)
        if self.density:
            lib().orc_collapse_dm(_ptr(self.a), self.n, q, outcome, p)
        else:
            lib().orc_collapse_sv(_ptr(self.a), self.n, q, outcome, p)
        return p

    def matrix(self):
        """Density matrix as a 2^N x 2^N array rho[j, k] = a[j + 2^N k]."""
        d = 1 << self.n
        return self.a.reshape(d, d).T


def run_circuit(n, ops, density=False):
    return State(n, density).run(ops)


def timed_run(n, ops, density=False):
    """Runs the gate list (allocation and |0> excluded from the timing, as in
    Sec. III); returns (state, seconds)."""
    s = State(n, density)
    t0 = time.perf_counter()
    s.run(ops)
    return s, time.perf_counter() - t0


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(t):
    """Host threads of the element-wise loops (results are unchanged)."""
    lib().orc_set_num_threads(int(t))
