"""calcInnerProduct / calcFidelity: FP64 reductions of <a|b> across
precisions, against exact host sums of the same amplitudes."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1802_08032_b300 import circuits as C
from gpu_helpers import PROB_TOL

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


def exact_inner(a, b):
    """sum conj(a) b, each part summed exactly (math.fsum)."""
    re = math.fsum((a.real * b.real).tolist() + (a.imag * b.imag).tolist())
    im = math.fsum((a.real * b.imag).tolist() + (-a.imag * b.real).tolist())
    return complex(re, im)


@pytest.mark.parametrize("pa,pb", [(128, 128), (128, 64), (64, 128), (64, 64)])
@pytest.mark.parametrize("n", [3, 11, 17])
def test_inner_product_matches_exact_host_sum(Q, env, pa, pb, n):
    qa = Q.createQureg(n, pa, env)
    qb = Q.createQureg(n, pb, env)
    try:
        Q.applyCircuit(qa, C.random_circuit(n, 8, 10 + n, extras=n >= 3))
        Q.applyCircuit(qb, C.random_circuit(n, 8, 20 + n, extras=n >= 3))
        z = Q.calcInnerProduct(qa, qb)
        f = Q.calcFidelity(qa, qb)
        a, b = Q.copyStateToHost(qa), Q.copyStateToHost(qb)
        # the same register against itself is its norm
        self_ip = Q.calcInnerProduct(qa, qa)
        tot = Q.calcTotalProb(qa)
    finally:
        Q.destroyQureg(qa)
        Q.destroyQureg(qb)
    want = exact_inner(a, b)
    assert abs(z - want) <= PROB_TOL
    assert abs(f - abs(want) ** 2) <= PROB_TOL
    assert abs(self_ip.imag) <= PROB_TOL and abs(self_ip.real - tot) <= PROB_TOL


def test_inner_product_against_oracle_states(Q, env):
    """complex128 registers: <a|b> equals the oracle's inner product of the
    oracle's states to the amplitude bar's order (1e-12)."""
    n = 12
    oa = C.random_circuit(n, 12, 5, extras=True)
    ob = C.random_circuit(n, 12, 6, extras=True)
    qa = Q.createQureg(n, 128, env)
    qb = Q.createQureg(n, 128, env)
    try:
        Q.applyCircuit(qa, oa)
        Q.applyCircuit(qb, ob)
        z = Q.calcInnerProduct(qa, qb)
    finally:
        Q.destroyQureg(qa)
        Q.destroyQureg(qb)
    want = exact_inner(O.run_circuit(n, oa).a, O.run_circuit(n, ob).a)
    assert abs(z - want) <= 1e-12


def test_inner_product_errors(Q, env):
    qa = Q.createQureg(5, 128, env)
    qb = Q.createQureg(6, 128, env)
    d = Q.createDensityQureg(3, 128, env)
    try:
        for x, y, name in ((qa, qb, "QS_E_QUBIT"), (qa, d, "QS_E_NOT_DENSITY")):
            with pytest.raises(Q.QSimError) as e:
                Q.calcInnerProduct(x, y)
            assert e.value.name == name
            with pytest.raises(Q.QSimError) as e:
                Q.calcFidelity(x, y)
            assert e.value.name == name
    finally:
        for q in (qa, qb, d):
            Q.destroyQureg(q)


# float32 values whose widening to FP64 has to be exact: normal ones of
# every size (taken by the integer-pipe widening), the smallest normal, and
# the ones that take the conversion instruction (subnormals, zeros)
EDGE_F32 = [1.0, -0.1, 3.0e-20, -1.17549435e-38, 1.0e-40, -1.4e-45, 1.5e18, 0.0, -0.0, 2.0 ** -126,
            0.7071067811865476, 123456.789]


@pytest.mark.parametrize("re", EDGE_F32)
def test_complex64_reductions_widen_exactly(Q, env, re):
    """One nonzero complex64 amplitude (re, im): the total probability is
    re^2 + im^2 rounded once (the FMA of im^2 onto the exact re^2; every
    other term adds zero), and <a|a> the same, for edge float32 values."""
    im = np.float32(-0.375)
    re32 = np.float32(re)
    a = np.zeros(1 << 4, dtype=np.complex64)
    a[5] = complex(re32, im)
    q = Q.createQureg(4, 64, env)
    try:
        Q.setAmps(q, a.astype(np.complex128))
        got = Q.calcTotalProb(q)
        want = float(np.float64(re32) ** 2 + np.float64(im) ** 2)   # re^2 exact in FP64, one rounding
        assert got == want, (re, got, want)
        ip = Q.calcInnerProduct(q, q)
        assert ip.real == want and ip.imag == 0.0
    finally:
        Q.destroyQureg(q)
