"""calcTotalProbNoAlloc, the allocation-free norm, against calcTotalProb.

The entry point serves callers that cannot allocate device memory (a host
framework that owns the device through its own pool, plug-ins given fixed
buffers): it takes caller-owned device input and output and keeps its scratch
in a fixed array inside the library.  This file is collected last, so a run
that stops at the first failure has run every other test before it.
"""
import math

import numpy as np
import pytest

from paper_1802_08032_b300 import circuits as C
from gpu_helpers import PROB_TOL

pytestmark = pytest.mark.gpu


def _prepared(Q, env, n, prec, seed):
    q = Q.createQureg(n, prec, env)
    Q.applyCircuit(q, C.random_circuit(n, 10, seed, extras=True))
    ref = Q.calcTotalProb(q)        # flushes and waits for the register's stream
    Q.syncQuESTEnv(env)
    return q, ref, Q.getQuregInfo(q)["devicePtr"]


def test_no_alloc_norm_matches_calc_total_prob_twice():
    import torch
    from paper_1802_08032_b300 import qsim as Q
    env = Q.createQuESTEnv()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")   # caller-owned output
    try:
        # two calls in a row: a larger array, then a smaller one, so stale
        # scratch from the first call would show up in the second
        qa, ref_a, ptr_a = _prepared(Q, env, 20, 128, 71)
        qb, ref_b, ptr_b = _prepared(Q, env, 15, 64, 72)
        stream = torch.cuda.current_stream()
        Q.calcTotalProbNoAlloc(ptr_a, 128, 1 << 20, out.data_ptr(), stream)
        Q.calcTotalProbNoAlloc(ptr_b, 64, 1 << 15, out.data_ptr() + 8, stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert abs(got[0] - ref_a) <= PROB_TOL
        assert abs(got[1] - ref_b) <= PROB_TOL
        # the same two calls again on a non-default stream give the same values
        s = torch.cuda.Stream()
        out2 = torch.zeros(2, dtype=torch.float64, device="cuda")
        Q.calcTotalProbNoAlloc(ptr_a, 128, 1 << 20, out2.data_ptr(), s)
        Q.calcTotalProbNoAlloc(ptr_b, 64, 1 << 15, out2.data_ptr() + 8, s)
        s.synchronize()
        assert np.array_equal(out2.cpu().numpy(), got)
        Q.destroyQureg(qa)
        Q.destroyQureg(qb)
    finally:
        Q.destroyQuESTEnv(env)


def test_no_alloc_norm_rejects_bad_sizes():
    import torch
    from paper_1802_08032_b300 import qsim as Q
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    amps = torch.zeros(64, dtype=torch.complex128, device="cuda")
    for n in (0, -5, (1 << 30) + 1):
        with pytest.raises(Q.QSimError) as e:
            Q.calcTotalProbNoAlloc(amps.data_ptr(), 128, n, out.data_ptr())
        assert e.value.name == "QS_E_ARG"
    with pytest.raises(Q.QSimError) as e:
        Q.calcTotalProbNoAlloc(amps.data_ptr(), 32, 64, out.data_ptr())
    assert e.value.name == "QS_E_ARG"
    # misaligned pointers are refused on the host, before anything launches
    for aptr, prec, optr in ((amps.data_ptr() + 8, 128, out.data_ptr()),
                             (amps.data_ptr() + 4, 64, out.data_ptr()),
                             (amps.data_ptr(), 128, out.data_ptr() + 4)):
        with pytest.raises(Q.QSimError) as e:
            Q.calcTotalProbNoAlloc(aptr, prec, 8, optr)
        assert e.value.name == "QS_E_ARG"
    amps[3] = 0.6 + 0.8j
    Q.calcTotalProbNoAlloc(amps.data_ptr(), 128, 64, out.data_ptr())
    torch.cuda.synchronize()
    assert abs(float(out[0]) - 1.0) <= PROB_TOL


@pytest.mark.parametrize("prec", [128, 64])
def test_no_alloc_norm_ragged_last_chunk(prec):
    """Several CTAs with a partial last chunk (3 * 16384 + 5 amplitudes) on a
    caller-filled array, against an exact host sum of the same values."""
    import torch
    from paper_1802_08032_b300 import qsim as Q
    n = 3 * 16384 + 5
    rng = np.random.default_rng(9)
    v = (rng.normal(size=n) + 1j * rng.normal(size=n)) * 1e-2
    dt = torch.complex128 if prec == 128 else torch.complex64
    amps = torch.from_numpy(v).to(dt).cuda()
    host = amps.cpu().numpy().astype(np.complex128)
    want = math.fsum((host.real ** 2).tolist() + (host.imag ** 2).tolist())
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        Q.calcTotalProbNoAlloc(amps.data_ptr(), prec, n, out.data_ptr())
        torch.cuda.synchronize()
        assert abs(float(out[0]) - want) <= PROB_TOL * max(1.0, want)
    # the same values in the first 3 * 16384 only: the tail's share is gone
    Q.calcTotalProbNoAlloc(amps.data_ptr(), prec, 3 * 16384, out.data_ptr())
    torch.cuda.synchronize()
    head = host[:3 * 16384]
    want_head = math.fsum((head.real ** 2).tolist() + (head.imag ** 2).tolist())
    assert abs(float(out[0]) - want_head) <= PROB_TOL * max(1.0, want_head)
