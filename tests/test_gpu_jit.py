"""Runtime-compiled pass kernels on the GPU: the same register run with the
interpreting fused kernel and with the generated kernels gives the same
amplitudes (bit for bit: the generated code applies the interpreter's own
arithmetic in the same order), and both match the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1802_08032_b300 import circuits as C
from gpu_helpers import AMP_TOL, PROB_TOL, gpu_state

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


def controlled_extras(n, seed):
    rng = C.SplitMix64(seed)
    ops = []
    for _ in range(2 * n):
        qs = C.distinct_qubits(rng, n, 3)
        a = C.haar_alpha_beta(rng)
        al, be = complex(a[0], a[1]), complex(a[2], a[3])
        u = (al.real, al.imag, -be.real, be.imag, be.real, be.imag, al.real, -al.imag)
        kind = rng.below(5)
        if kind == 0:
            ops.append(C.Op("CNOT", (qs[0],), (qs[1],)))
        elif kind == 1:
            ops.append(C.Op("CUNITARY", (qs[0],), tuple(qs[1:]), u))
        elif kind == 2:
            ops.append(C.Op("PHASE", (qs[0],), (), (0.3 + rng.uniform(),)))
        elif kind == 3:
            ops.append(C.Op("X", (qs[0],)))
        else:
            ops.append(C.Op("UNITARY", (qs[0],), (), u))
    return ops


def run_both(Q, env, n, ops, prec, arith=0, density=False, tile=0, min_q=None, copy=0, ctas=2, direct=0,
             swizzle=1):
    """(interpreted, compiled) final states; checks the compiled run really
    launched generated kernels and none failed.  copy = 1 / 2: the bulk-copy
    (TMA) / async-copy pipeline forms of the generated kernels."""
    Q.setEnvOption(env, "arith", arith)
    Q.setEnvOption(env, "tile_qubits", tile)
    Q.setEnvOption(env, "jit_fp64", 1)
    Q.setEnvOption(env, "jit_copy", copy)
    Q.setEnvOption(env, "jit_ctas", ctas)
    Q.setEnvOption(env, "jit_direct", direct)
    Q.setEnvOption(env, "jit_swizzle", swizzle)
    # a single-tile register would otherwise run on a thread-block cluster
    # (the interpreting cluster kernel), which generated kernels do not replace
    Q.setEnvOption(env, "fused_cluster", 0)
    if min_q is not None:
        Q.setEnvOption(env, "jit_min_qubits", min_q)
    try:
        Q.setEnvOption(env, "jit", 0)
        a = gpu_state(Q, env, n, ops, prec, density=density)
        Q.setEnvOption(env, "jit", 1)
        l0 = Q.getEnvOption(env, "jit_launches")
        b = gpu_state(Q, env, n, ops, prec, density=density)
        launched = Q.getEnvOption(env, "jit_launches") - l0
    finally:
        Q.setEnvOption(env, "jit", 2)
        Q.setEnvOption(env, "jit_fp64", 0)
        Q.setEnvOption(env, "jit_copy", -1)
        Q.setEnvOption(env, "jit_ctas", 0)
        Q.setEnvOption(env, "jit_direct", 1)
        Q.setEnvOption(env, "jit_swizzle", 1)
        Q.setEnvOption(env, "arith", 0)
        Q.setEnvOption(env, "tile_qubits", 0)
        Q.setEnvOption(env, "jit_min_qubits", 20)
        Q.setEnvOption(env, "fused_cluster", 8)
    assert Q.getEnvOption(env, "jit_failed") == 0
    assert Q.getEnvOption(env, "jit_rejected") == 0
    assert launched > 0
    return a, b


@pytest.mark.parametrize("copy,direct", [(0, 0), (1, 0), (2, 0), (0, 1), (2, 1)])
@pytest.mark.parametrize("prec,arith", [(64, 0), (128, 0), (128, 1)])
@pytest.mark.parametrize("n", [12, 21])
def test_compiled_passes_match_interpreter_and_oracle(Q, env, prec, arith, n, copy, direct):
    ops = C.random_circuit(n, 14, 900 + n, extras=True)
    ops = ops[: len(ops) // 2] + controlled_extras(n, n) + ops[len(ops) // 2:]
    a, b = run_both(Q, env, n, ops, prec, arith, min_q=1, copy=copy, direct=direct)
    assert np.array_equal(a, b), float(np.max(np.abs(a - b)))
    ref = O.run_circuit(n, ops).a
    assert np.max(np.abs(b - ref)) <= AMP_TOL[prec]


@pytest.mark.parametrize("copy,ctas,direct,swizzle", [(0, 2, 0, 1), (1, 3, 0, 1), (2, 3, 0, 1), (2, 3, 1, 1),
                                                      (0, 2, 1, 1), (2, 3, 1, 0)])
@pytest.mark.parametrize("prec,arith", [(64, 0), (128, 0), (128, 1)])
@pytest.mark.parametrize("tile", [9, 11])
def test_compiled_passes_with_small_tiles(Q, env, prec, arith, tile, copy, ctas, direct, swizzle):
    """Tiles smaller than the register: conditions on global bits (the tile
    base) and on local bits outside the stage's register bits; with the
    bulk-copy pipeline, several tiles per CTA (both buffers in turn)."""
    n = 15
    ops = C.random_circuit(n, 12, 77 + tile, extras=True) + controlled_extras(n, tile)
    ops = ops[len(ops) // 4:]  # a suffix: phases land on qubits outside the first tile
    a, b = run_both(Q, env, n, ops, prec, arith, tile=tile, min_q=1, copy=copy, ctas=ctas, direct=direct,
                    swizzle=swizzle)
    assert np.array_equal(a, b), float(np.max(np.abs(a - b)))
    ref = O.run_circuit(n, ops).a
    assert np.max(np.abs(b - ref)) <= AMP_TOL[prec]


@pytest.mark.parametrize("copy,direct", [(0, 0), (1, 0), (2, 0), (2, 1)])
@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("p", [(0.01, 0.005), (0.3, 0.6)])
def test_compiled_density_matrix(Q, env, arith, p, copy, direct):
    N = 7
    ops = C.with_noise(C.random_circuit(N, 10, 31, extras=True) + controlled_extras(N, 3), *p)
    a, b = run_both(Q, env, N, ops, 128, arith, density=True, min_q=1, copy=copy, direct=direct)
    assert np.array_equal(a, b), float(np.max(np.abs(a - b)))
    ref = O.run_circuit(N, ops, density=True).a
    assert np.max(np.abs(b - ref)) <= AMP_TOL[128]


@pytest.mark.parametrize("copy,tile,direct", [(0, 0, 0), (1, 12, 0), (2, 12, 0), (2, 13, 0), (-1, 0, 0),
                                              (-1, 0, 1)])
def test_compiled_26_qubit_workload_reductions(Q, env, copy, tile, direct):
    """The depth-40 workload layering at 26 qubits (default threshold, so the
    generated kernels are the ones a user gets): complex64 amplitudes and FP64
    reductions equal to the interpreted run's."""
    n = 26
    ops = C.workload_30q(n)
    out = []
    Q.setEnvOption(env, "jit_copy", copy)
    Q.setEnvOption(env, "tile_qubits", tile)
    Q.setEnvOption(env, "jit_ctas", 3 if tile == 12 else (1 if copy > 0 else 0))
    Q.setEnvOption(env, "jit_direct", direct)
    for jit in (0, 1):
        Q.setEnvOption(env, "jit", jit)
        q = Q.createQureg(n, 64, env)
        try:
            Q.applyCircuit(q, ops)
            tot = Q.calcTotalProb(q)
            p = Q.calcProbOfOutcome(q, 7, 1)
            amps = Q.copyStateToHost(q, 0, 1 << 16)
        finally:
            Q.destroyQureg(q)
        out.append((tot, p, amps))
    Q.setEnvOption(env, "jit", 2)
    Q.setEnvOption(env, "jit_copy", -1)
    Q.setEnvOption(env, "tile_qubits", 0)
    Q.setEnvOption(env, "jit_ctas", 0)
    Q.setEnvOption(env, "jit_direct", 1)
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2])
    assert abs(out[1][0] - 1) <= 1e-5


def test_background_compile_then_reuse(Q, env):
    """Option 2: a pass structure met for the first time runs on the
    interpreting kernel and is not compiled; met again, it is compiled in the
    background while the interpreting kernel runs it.  Once compiled, the same circuit
    structure with other angles launches only cached kernels (coefficients
    are kernel parameters, not part of the compiled code) and matches the
    oracle."""
    n = 20

    def circuit(seed):
        ops = C.random_circuit(n, 8, 4321, extras=False)
        r = C.SplitMix64(seed)
        return ops + [C.Op("PHASE", (q,), (), (0.2 + 0.2 * r.uniform(),)) for q in range(n)] + \
            [C.Op("H", (q,)) for q in range(n)]

    def counted(ops, jit):
        Q.setEnvOption(env, "jit", jit)
        l0, p0 = Q.getEnvOption(env, "jit_launches"), Q.getEnvOption(env, "fused_passes")
        st = gpu_state(Q, env, n, ops, 64)
        return st, Q.getEnvOption(env, "jit_launches") - l0, Q.getEnvOption(env, "fused_passes") - p0

    try:
        _, jl, passes = counted(circuit(1), 2)
        assert passes > 0 and jl == 0        # nothing compiled yet: all interpreted
        known = Q.getEnvOption(env, "jit_pending") + Q.getEnvOption(env, "jit_ready")
        _, jl, passes = counted(circuit(1), 2)  # met a second time: queued, still interpreted
        assert Q.getEnvOption(env, "jit_pending") + Q.getEnvOption(env, "jit_ready") > known
        _, jl, passes = counted(circuit(1), 1)
        assert jl == passes                   # waited for the compiles
        ops = circuit(2)
        got, jl, passes = counted(ops, 2)
        assert jl == passes                   # other angles: the cached kernels
    finally:
        Q.setEnvOption(env, "jit", 2)
    ref = O.run_circuit(n, ops).a
    assert np.max(np.abs(got - ref)) <= AMP_TOL[64]
