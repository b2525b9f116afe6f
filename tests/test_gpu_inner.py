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
