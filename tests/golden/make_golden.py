"""Writes the full-size expected values used by the GPU parity tests.

Calls only the CPU oracle (oracle/) and the seeded generator; no value here
comes from the CUDA path.  Each fixture stores the gate-list hash it was
computed for, the reductions, and the amplitudes at seeded sample indices.

  python tests/golden/make_golden.py dm14     # 14-qubit noisy density matrix
  python tests/golden/make_golden.py sv33emb  # factors of a 33-qubit product state
  python tests/golden/make_golden.py sv30     # 30-qubit complex128, depth 40 (~1-2 h on 8 cores)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1802_08032_b300 import circuits as C  # noqa: E402

SAMPLES = 4096


def amps_at(state, idx):
    return [[float(state.a[i].real), float(state.a[i].imag)] for i in idx]


def sv30():
    n = 30
    ops = C.workload_30q(n)
    t0 = time.time()
    s = O.run_circuit(n, ops)
    idx = C.sample_indices(n, SAMPLES, 30)
    out = {"what": "30-qubit complex128 state vector after the seeded depth-40 random circuit "
                   "(layering with per-layer compactUnitary and 3-control phase flip), CPU oracle",
           "qubits": n, "ops": len(ops), "hash": C.stream_hash(ops),
           "total_prob": s.total_prob(),
           "prob_outcome_1": [s.prob_outcome(q, 1) for q in range(n)],
           "indices": idx, "amps": amps_at(s, idx), "oracle_seconds": time.time() - t0}
    return "sv30_depth40.json", out


def dm14():
    N = 14
    ops = C.workload_dm14(N)
    t0 = time.time()
    s = O.run_circuit(N, ops, density=True)
    idx = C.sample_indices(2 * N, SAMPLES, 14)
    d = 1 << N
    diag = sorted(set(C.sample_indices(N, 256, 41)))
    out = {"what": "14-qubit density matrix after the seeded depth-20 random circuit with "
                   "mixDephasing(0.01) then mixDepolarising(0.005) on every gate qubit, CPU oracle",
           "qubits": N, "ops": len(ops), "hash": C.stream_hash(ops),
           "trace": s.total_prob(), "purity": s.purity(),
           "prob_outcome_1": [s.prob_outcome(q, 1) for q in range(N)],
           "indices": idx, "amps": amps_at(s, idx),
           "diag_rows": diag, "diag": amps_at(s, [j + d * j for j in diag]),
           "oracle_seconds": time.time() - t0}
    return "dm14_depth20.json", out


def sv33emb():
    """33 qubits as a product: a 30-qubit circuit on qubits 0..29 and a
    3-qubit circuit on qubits 30..32.  Stores both factors' amplitudes at
    sample indices so the 33-qubit amplitudes are products of the two."""
    a_ops = C.random_circuit(30, 12, 3330, extras=True)
    b_ops = C.random_circuit(3, 12, 3333, extras=True)
    t0 = time.time()
    a = O.run_circuit(30, a_ops)
    b = O.run_circuit(3, b_ops)
    idx = C.sample_indices(30, SAMPLES, 33)
    out = {"what": "factors of a 33-qubit product state: 30-qubit depth-12 circuit on qubits "
                   "0..29 (seed 3330) and 3-qubit depth-12 circuit on qubits 30..32 (seed 3333)",
           "hash_low": C.stream_hash(a_ops), "hash_high": C.stream_hash(b_ops),
           "low_indices": idx, "low_amps": amps_at(a, idx),
           "high_amps": amps_at(b, list(range(8))),
           "low_total_prob": a.total_prob(),
           "low_prob_outcome_1": [a.prob_outcome(q, 1) for q in range(30)],
           "high_prob_outcome_1": [b.prob_outcome(q, 1) for q in range(3)],
           "oracle_seconds": time.time() - t0}
    return "sv33_product_factors.json", out


if __name__ == "__main__":
    for what in sys.argv[1:]:
        name, data = {"sv30": sv30, "dm14": dm14, "sv33emb": sv33emb}[what]()
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(data, f)
        print(name, "written", f"{data['oracle_seconds']:.0f} s", flush=True)
