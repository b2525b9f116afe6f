"""Seeded synthetic workloads: random circuits as plain gate lists.

This module draws random numbers and lays gates out; it holds no gate
arithmetic (no matrices, no amplitudes).  Both the CUDA path and the CPU
oracle consume its output, and each side builds its own gate matrices.

Workload (the paper's benchmark is random circuits over the universal set
{H, T, CZ, X^1/2, Y^1/2}, Sec. II.C).  The generator the paper uses is not
reproduced in the paper, so the layering below is this library's reading:

* layer 0: H on every qubit;
* layer l >= 1: CZ on (i, i+1) for every i = (l-1) mod 2 (step 2, i+1 < n),
  then one gate drawn uniformly from {sqrt(X), sqrt(Y), T} on every qubit
  i = l mod 2 (step 2)   ("alternate" layering);
* optional per-layer extras (l >= 1): compactUnitary with Haar-random
  (alpha, beta) on one uniform qubit, then multiControlledPhaseFlip on three
  distinct uniform qubits;
* density-matrix circuits: after every gate, mixDephasing then
  mixDepolarising on each qubit the gate acts on (both qubits of a CZ).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), doubles as (x >> 11) * 2^-53
and Gaussians by the Box-Muller transform.
"""
from __future__ import annotations

import hashlib
import math
import struct
from typing import List, NamedTuple, Sequence, Tuple

MASK64 = (1 << 64) - 1

# Gate kinds.  Matrices are NOT defined here: each consumer defines them.
H, SQRT_X, SQRT_Y, T_GATE, PHASE = "H", "SX", "SY", "T", "PHASE"
CZ, CNOT, X_GATE = "CZ", "CNOT", "X"
COMPACT, UNITARY, CUNITARY, MCPF = "COMPACT", "UNITARY", "CUNITARY", "MCPF"
DEPHASE, DEPOL = "DEPHASE", "DEPOL"

KINDS = (H, SQRT_X, SQRT_Y, T_GATE, PHASE, CZ, CNOT, X_GATE, COMPACT, UNITARY,
         CUNITARY, MCPF, DEPHASE, DEPOL)
CHANNELS = (DEPHASE, DEPOL)


class Op(NamedTuple):
    """One call of the library's API.

    kind     : one of KINDS
    targets  : qubits acted on (CZ: both qubits; MCPF: empty)
    controls : control qubits (CNOT/CUNITARY: one; MCPF: all of them)
    params   : floats (COMPACT: a.re, a.im, b.re, b.im;  UNITARY/CUNITARY:
               8 floats, row-major u00 u01 u10 u11 as (re, im);
               DEPHASE/DEPOL: (p,))
    """
    kind: str
    targets: Tuple[int, ...] = ()
    controls: Tuple[int, ...] = ()
    params: Tuple[float, ...] = ()

    def qubits(self) -> Tuple[int, ...]:
        return tuple(self.targets) + tuple(self.controls)


class SplitMix64:
    """SplitMix64 generator (Steele, Lea, Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (2.0 ** -53)

    def below(self, m: int) -> int:
        """Integer in [0, m): floor(u * m) with u a 53-bit uniform."""
        return ((self.next_u64() >> 11) * m) >> 53

    def gauss_pair(self) -> Tuple[float, float]:
        """Two independent N(0, 1) draws (Box-Muller)."""
        u1 = 1.0 - self.uniform()          # (0, 1]: log is finite
        u2 = self.uniform()
        r = math.sqrt(-2.0 * math.log(u1))
        return r * math.cos(2.0 * math.pi * u2), r * math.sin(2.0 * math.pi * u2)


def haar_alpha_beta(rng: SplitMix64) -> Tuple[float, float, float, float]:
    """Haar-random SU(2) column (alpha, beta): a normalised complex Gaussian
    2-vector, returned as (alpha.re, alpha.im, beta.re, beta.im)."""
    g0, g1 = rng.gauss_pair()
    g2, g3 = rng.gauss_pair()
    r = math.sqrt(g0 * g0 + g1 * g1 + g2 * g2 + g3 * g3)
    return (g0 / r, g1 / r, g2 / r, g3 / r)


def distinct_qubits(rng: SplitMix64, n: int, k: int) -> Tuple[int, ...]:
    """k distinct uniform qubits in [0, n), in draw order (rejection)."""
    out: List[int] = []
    while len(out) < k:
        q = rng.below(n)
        if q not in out:
            out.append(q)
    return tuple(out)


def random_circuit(n: int, depth: int, seed: int, extras: bool = False,
                   layering: str = "alternate") -> List[Op]:
    """Seeded random circuit on n qubits with `depth` layers (layer 0 = H).

    layering="alternate": singles on qubits i = l mod 2 (the default reading).
    layering="free": singles on the qubits that no CZ of this layer touches.
    """
    if n < 1 or depth < 1:
        raise ValueError("need n >= 1 and depth >= 1")
    if extras and n < 3:
        raise ValueError("extras need n >= 3 (three distinct controls)")
    rng = SplitMix64(seed)
    singles = (SQRT_X, SQRT_Y, T_GATE)
    ops: List[Op] = [Op(H, (q,)) for q in range(n)]
    for layer in range(1, depth):
        cz_start = (layer - 1) % 2
        busy = set()
        for i in range(cz_start, n - 1, 2):
            ops.append(Op(CZ, (i, i + 1)))
            busy.update((i, i + 1))
        if layering == "alternate":
            sq = range(layer % 2, n, 2)
        elif layering == "free":
            sq = [q for q in range(n) if q not in busy]
        else:
            raise ValueError(f"unknown layering {layering!r}")
        for q in sq:
            ops.append(Op(singles[rng.below(3)], (q,)))
        if extras:
            q = rng.below(n)
            ops.append(Op(COMPACT, (q,), (), haar_alpha_beta(rng)))
            ops.append(Op(MCPF, (), distinct_qubits(rng, n, 3)))
    return ops


def with_noise(ops: Sequence[Op], p_dephase: float, p_depol: float) -> List[Op]:
    """Density-matrix workload: after every gate, mixDephasing(p_dephase) then
    mixDepolarising(p_depol) on each qubit the gate acts on."""
    out: List[Op] = []
    for op in ops:
        out.append(op)
        if op.kind in CHANNELS:
            continue
        for q in op.qubits():
            if p_dephase > 0:
                out.append(Op(DEPHASE, (q,), (), (p_dephase,)))
            if p_depol > 0:
                out.append(Op(DEPOL, (q,), (), (p_depol,)))
    return out


def random_density_circuit(N: int, depth: int, seed: int, p_dephase: float,
                           p_depol: float) -> List[Op]:
    return with_noise(random_circuit(N, depth, seed), p_dephase, p_depol)


def serialize(ops: Sequence[Op]) -> bytes:
    """Canonical byte form of a gate list (floats as exact IEEE bits)."""
    out = bytearray()
    for op in ops:
        out += op.kind.encode() + b"|"
        out += ",".join(map(str, op.targets)).encode() + b"|"
        out += ",".join(map(str, op.controls)).encode() + b"|"
        out += b"".join(struct.pack("<d", float(p)) for p in op.params) + b"\n"
    return bytes(out)


def stream_hash(ops: Sequence[Op]) -> str:
    return hashlib.sha256(serialize(ops)).hexdigest()


def sample_indices(nq: int, count: int, seed: int) -> List[int]:
    """Seeded sample of amplitude indices in [0, 2^nq), always including the
    first and the last index."""
    rng = SplitMix64(seed)
    dim = 1 << nq
    idx = {0, dim - 1}
    while len(idx) < min(count, dim):
        idx.add(rng.next_u64() & (dim - 1))
    return sorted(idx)


# Named workloads (sizes of the paper-style benchmark configurations).
def workload_12q():
    return random_circuit(12, 20, 1802)


def workload_30q(n: int = 30):
    return random_circuit(n, 40, 8032, extras=True)


def workload_dm14(N: int = 14):
    return random_density_circuit(N, 20, 14, 0.01, 0.005)
