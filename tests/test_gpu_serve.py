"""Serving loop: results against the CPU oracle, alone vs in the mix,
admission under a memory budget, bounded polls, invalid requests."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1802_08032_b300 import circuits as C
from gpu_helpers import AMP_TOL, PROB_TOL

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


def mixed_requests(count, seed):
    """(kind, n, prec, ops) like the serving workload, at sizes the oracle
    finishes quickly: state vectors 4..14 qubits (c64 or c128), density
    matrices 2..6 qubits (c64 or c128) with dephasing 0.01."""
    rng = C.SplitMix64(seed)
    reqs = []
    for i in range(count):
        kind = rng.below(3)
        depth = 4 + rng.below(10)
        if kind == 2:
            N = 2 + rng.below(5)
            ops = C.with_noise(C.random_circuit(N, depth, seed + i), 0.01, 0.0)
            reqs.append((True, N, 64 if rng.below(2) == 0 else 128, ops))
        else:
            n = 4 + rng.below(11)
            reqs.append((False, n, 64 if kind == 0 else 128,
                         C.random_circuit(n, depth, seed + i, extras=n >= 3)))
    return reqs


def run_all(Q, srv, reqs, want_amps=True):
    tickets, bufs = [], []
    for dens, n, prec, ops in reqs:
        nq = 2 * n if dens else n
        buf = np.empty(1 << nq, dtype=np.complex128) if want_amps else None
        tickets.append(Q.serveSubmit(srv, ops, n, prec, dens, measureQubit=n - 1, outAmps=buf))
        bufs.append(buf)
    return [Q.servePoll(srv, t) for t in tickets], bufs


def test_serving_matches_oracle(Q, env):
    reqs = mixed_requests(40, 5000)
    srv = Q.serveCreate(env, slots=8, budgetBytes=1 << 30)
    try:
        results, bufs = run_all(Q, srv, reqs)
    finally:
        Q.serveDestroy(srv)
    for (dens, n, prec, ops), res, buf in zip(reqs, results, bufs):
        assert res["status"] == 0
        ref = O.run_circuit(n, ops, density=dens)
        assert np.max(np.abs(buf - ref.a)) <= AMP_TOL[prec]
        tol = PROB_TOL if prec == 128 else 1e-5
        assert abs(res["totalProb"] - ref.total_prob()) <= tol
        assert abs(res["probOutcome0"] - ref.prob_outcome(n - 1, 0)) <= tol
        assert res["latencyUs"] >= res["queuedUs"] >= 0


def test_results_same_alone_and_in_the_mix(Q, env):
    """One slot, one request at a time, against eight slots with every
    request submitted at once: the same kernels on the same data, so the
    results agree bit for bit."""
    reqs = mixed_requests(24, 6000)
    alone = Q.serveCreate(env, slots=1, budgetBytes=1 << 30)
    try:
        ra, ba = [], []
        for r in reqs:
            res, buf = run_all(Q, alone, [r])
            ra += res
            ba += buf
    finally:
        Q.serveDestroy(alone)
    mix = Q.serveCreate(env, slots=8, budgetBytes=1 << 30)
    try:
        rm, bm = run_all(Q, mix, reqs)
    finally:
        Q.serveDestroy(mix)
    assert len({r["slot"] for r in rm}) > 1          # they really ran on several slots
    for a, m, x, y in zip(ra, rm, ba, bm):
        assert a["totalProb"] == m["totalProb"] and a["probOutcome0"] == m["probOutcome0"]
        assert np.array_equal(x, y)


def test_budget_admission_and_rejection(Q, env):
    # budget for two 16-qubit complex128 registers (1 MiB each) at a time
    srv = Q.serveCreate(env, slots=8, budgetBytes=2 << 20)
    try:
        ops = C.random_circuit(16, 6, 42, extras=True)
        ts = [Q.serveSubmit(srv, ops, 16, 128) for _ in range(6)]
        res = [Q.servePoll(srv, t) for t in ts]
        assert all(r["status"] == 0 for r in res)
        assert all(abs(r["totalProb"] - 1) <= PROB_TOL for r in res)
        with pytest.raises(Q.QSimError) as e:         # larger than the whole budget
            Q.serveSubmit(srv, C.random_circuit(18, 2, 1), 18, 128)
        assert e.value.name == "QS_E_NOMEM"
    finally:
        Q.serveDestroy(srv)


def test_invalid_requests_and_bounded_poll(Q, env):
    srv = Q.serveCreate(env, slots=2, budgetBytes=1 << 30)
    try:
        with pytest.raises(Q.QSimError) as e:
            Q.serveSubmit(srv, [C.Op("H", (7,))], 5, 64)
        assert e.value.name == "QS_E_QUBIT"
        with pytest.raises(Q.QSimError) as e:
            Q.serveSubmit(srv, [C.Op("DEPHASE", (0,), (), (0.1,))], 5, 64)
        assert e.value.name == "QS_E_NOT_DENSITY"
        big = C.random_circuit(24, 40, 9, extras=True)      # keeps the GPU busy for a while
        t = Q.serveSubmit(srv, big, 24, 128)
        with pytest.raises(Q.QSimError) as e:
            Q.servePoll(srv, t, timeoutUs=0)
        assert e.value.name == "QS_E_TIMEOUT"
        ok = Q.servePoll(srv, t)
        assert ok["status"] == 0 and abs(ok["totalProb"] - 1) <= PROB_TOL
        with pytest.raises(Q.QSimError) as e:            # a ticket is collected once
            Q.servePoll(srv, t, timeoutUs=0)
        assert e.value.name == "QS_E_HANDLE"
    finally:
        Q.serveDestroy(srv)


def test_admission_policy_sheds_and_refuses(Q, env):
    """Past saturation: with a queue-wait bound, requests stuck behind a long
    one are shed (QS_E_BUSY) instead of waiting; with a queue-length bound,
    submissions are refused while the queue is full.  The long request and
    the ones admitted in time still complete correctly."""
    long_ops = C.random_circuit(27, 40, 77, extras=True)
    short = [C.random_circuit(10, 6, 900 + i) for i in range(6)]
    srv = Q.serveCreate(env, slots=1, budgetBytes=1 << 34)
    try:
        Q.serveSetOption(srv, "max_queue_us", 20_000)
        t_long = Q.serveSubmit(srv, long_ops, 27, 128)
        ts = [Q.serveSubmit(srv, ops, 10, 64) for ops in short]
        r_long = Q.servePoll(srv, t_long, timeoutUs=120_000_000)
        rs = [Q.servePoll(srv, t, timeoutUs=120_000_000) for t in ts]
        assert r_long["status"] == 0 and abs(r_long["totalProb"] - 1) <= PROB_TOL
        names = [Q.ERRORS[r["status"]] for r in rs]
        assert "QS_E_BUSY" in names, names
        assert Q.serveGetOption(srv, "shed") == names.count("QS_E_BUSY")
        for r, ops in zip(rs, short):
            if r["status"] == 0:
                assert abs(r["totalProb"] - 1) <= 1e-5
            else:
                assert r["slot"] == -1 and r["queuedUs"] >= 20_000
        # back-pressure: two may wait, the third is refused at submission
        Q.serveSetOption(srv, "max_queue_us", 0)
        Q.serveSetOption(srv, "max_queue", 2)
        t_long = Q.serveSubmit(srv, long_ops, 27, 128)
        import time
        deadline = time.time() + 30
        while Q.serveGetOption(srv, "queued") > 0 and time.time() < deadline:
            time.sleep(0.001)          # the long one is admitted (leaves the queue)
        t1 = Q.serveSubmit(srv, short[0], 10, 64)
        t2 = Q.serveSubmit(srv, short[1], 10, 64)
        if Q.serveGetOption(srv, "queued") == 2:
            with pytest.raises(Q.QSimError) as e:
                Q.serveSubmit(srv, short[2], 10, 64)
            assert e.value.name == "QS_E_BUSY"
            assert Q.serveGetOption(srv, "refused") == 1
        for t in (t_long, t1, t2):
            assert Q.servePoll(srv, t, timeoutUs=120_000_000)["status"] == 0
        with pytest.raises(Q.QSimError) as e:
            Q.serveSetOption(srv, "max_queue", -1)
        assert e.value.name == "QS_E_ARG"
    finally:
        Q.serveDestroy(srv)
