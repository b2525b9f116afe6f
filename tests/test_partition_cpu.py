"""Partitioned state vectors on the CPU (no GPU): the swap schedule the
library plans (partPlanSchedule, host-only C ABI) executed on 2^k slices of
a state, once in one process and once as gloo ranks exchanging half-slices
with point-to-point sends, against the oracle's full state.  A rank that
leaves between steps is detected by its partner's next exchange.

The paper distributes the state vector over 2^k nodes by its top k index
bits (Sec. II.B.2); a gate on a qubit held in the node index needs data from
the pair node.  The library swaps such a qubit with a local one first (each
pair exchanges half of its amplitudes).  Here the local gate application on
a slice is the oracle's (test infrastructure); the schedule, the qubit map
and the exchange pattern are the library's.
"""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_1802_08032_b300 import circuits as C
from paper_1802_08032_b300 import qsim as Q

MOVING = ("H", "X", "SX", "SY", "COMPACT", "UNITARY", "CNOT", "CUNITARY")


def circuit(n, seed):
    """Random layering plus gates on every qubit (so every global qubit is
    moved at least once) and controls on high qubits."""
    rng = C.SplitMix64(seed)
    ops = C.random_circuit(n, 6, seed, extras=True)
    for q in range(n):
        ops.append(C.Op("H", (q,)))
        c = (q + n - 1) % n
        ops.append(C.Op("CNOT", (q,), (c,)))
        a = C.haar_alpha_beta(rng)
        ops.append(C.Op("COMPACT", (n - 1 - q,), (), a))
    ops.append(C.Op("MCPF", (), (n - 1, n - 2, 0)))
    ops.append(C.Op("PHASE", (n - 1,), (), (0.7,)))
    return ops


def apply_local(vec, op, perm, m, part):
    """The gate `op` as part `part` applies it to its slice `vec` (m local
    qubits) under the logical -> physical map `perm`; returns the slice."""
    bit = lambda phys: (part >> (phys - m)) & 1  # noqa: E731
    st = O.State(m, amps=vec)
    k = op.kind
    if k in MOVING:
        ctr = []
        for c in op.controls:
            p = perm[c]
            if p >= m:
                if not bit(p):
                    return vec
            else:
                ctr.append(p)
        t = perm[op.targets[0]]
        assert t < m, "moved qubit not local"
        st.gate(t, O.gate_matrix(k, op.params), tuple(ctr))
        return st.a
    if k in ("T", "PHASE"):
        t = perm[op.targets[0]]
        if t < m:
            st.gate(t, O.gate_matrix(k, op.params))
            return st.a
        return vec * O.gate_matrix(k, op.params)[1, 1] if bit(t) else vec
    if k in ("CZ", "MCPF"):
        qs = op.targets if k == "CZ" else op.controls
        loc = []
        for q in qs:
            p = perm[q]
            if p >= m:
                if not bit(p):
                    return vec
            else:
                loc.append(p)
        if not loc:
            return -vec
        st.phase_flip(tuple(loc))
        return st.a
    raise AssertionError(k)


def halves(vec, l):
    return vec.reshape(-1, 2, 1 << l)


def run_schedule_in_process(n, k, ops):
    steps, final_perm = Q.partPlanSchedule(n, k, ops)
    m = n - k
    slices = [np.zeros(1 << m, complex) for _ in range(1 << k)]
    slices[0][0] = 1
    perm = list(range(n))
    for kind, oi, g, l in steps:
        if kind == 1:
            b = 1 << (g - m)
            for p0 in range(1 << k):
                if p0 & b:
                    continue
                a, c = halves(slices[p0], l), halves(slices[p0 | b], l)
                tmp = a[:, 1, :].copy()
                a[:, 1, :] = c[:, 0, :]
                c[:, 0, :] = tmp
            lq, gq = perm.index(l), perm.index(g)
            perm[lq], perm[gq] = g, l
        else:
            for p in range(1 << k):
                slices[p] = apply_local(slices[p], ops[oi], perm, m, p)
    assert perm == final_perm
    return unpermute(np.concatenate(slices), perm, n)


def unpermute(phys, perm, n):
    idx = np.arange(1 << n)
    logical = np.zeros_like(idx)
    for q in range(n):
        logical |= ((idx >> perm[q]) & 1) << q
    out = np.empty_like(phys)
    out[logical] = phys
    return out


@pytest.mark.parametrize("n,k", [(6, 1), (7, 2), (9, 3), (10, 2)])
def test_schedule_keeps_moved_qubits_local(n, k):
    ops = circuit(n, 40 + n)
    steps, final_perm = Q.partPlanSchedule(n, k, ops)
    m = n - k
    perm = list(range(n))
    local_ops = 0
    for kind, oi, g, l in steps:
        if kind == 1:
            assert g >= m and l < m
            lq, gq = perm.index(l), perm.index(g)
            perm[lq], perm[gq] = g, l
        else:
            op = ops[oi]
            assert oi == local_ops
            local_ops += 1
            if op.kind in MOVING:
                assert perm[op.targets[0]] < m
    assert local_ops == len(ops) and perm == final_perm
    assert sorted(final_perm) == list(range(n))
    # a swap happens only for a gate on a global qubit
    assert 0 < sum(1 for s in steps if s[0] == 1) <= len(ops)


@pytest.mark.parametrize("n,k", [(6, 1), (7, 2), (9, 3), (11, 2)])
def test_schedule_reproduces_the_oracle(n, k):
    ops = circuit(n, 70 + n)
    got = run_schedule_in_process(n, k, ops)
    want = O.run_circuit(n, ops).a
    assert np.max(np.abs(got - want)) <= 1e-12


def test_diagonal_and_controlled_gates_need_no_swap():
    """Phases, sign flips and controls on global qubits never trigger an
    exchange (a part knows its global bits)."""
    n, k = 8, 2
    ops = [C.Op("H", (q,)) for q in range(6)] + [
        C.Op("T", (7,)), C.Op("CZ", (6, 7)), C.Op("MCPF", (), (7, 6, 1)),
        C.Op("CNOT", (2,), (7,)), C.Op("PHASE", (6,), (), (0.3,))]
    steps, _ = Q.partPlanSchedule(n, k, ops)
    assert all(s[0] == 0 for s in steps)
    got = run_schedule_in_process(n, k, ops)
    assert np.max(np.abs(got - O.run_circuit(n, ops).a)) <= 1e-13


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, n, seed, leave_after, out):
    """One part per gloo rank: local gates on the rank's slice, swaps as
    half-slice exchanges with the partner rank (isend + recv)."""
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    k = world.bit_length() - 1
    m = n - k
    ops = circuit(n, seed)
    steps, final_perm = Q.partPlanSchedule(n, k, ops)
    vec = np.zeros(1 << m, complex)
    if rank == 0:
        vec[0] = 1
    perm = list(range(n))
    swaps = 0
    try:
        for si, (kind, oi, g, l) in enumerate(steps):
            if kind == 1:
                if leave_after is not None and swaps == leave_after and rank == 1:
                    out[rank] = "left"
                    os._exit(0)                     # leaves between steps, nothing in flight
                b = (rank >> (g - m)) & 1
                partner = rank ^ (1 << (g - m))
                h = halves(vec, l)
                send = torch.from_numpy(np.ascontiguousarray(h[:, 1 - b, :])).view(torch.float64).reshape(-1)
                recv = torch.empty_like(send)
                req = dist.isend(send, partner)
                dist.recv(recv, partner)
                req.wait()
                h[:, 1 - b, :] = recv.view(torch.complex128).numpy().reshape(h[:, 1 - b, :].shape)
                lq, gq = perm.index(l), perm.index(g)
                perm[lq], perm[gq] = g, l
                swaps += 1
            else:
                vec = apply_local(vec, ops[oi], perm, m, rank)
        assert perm == final_perm
        flat = torch.from_numpy(np.ascontiguousarray(vec)).view(torch.float64)
        parts = [torch.empty_like(flat) for _ in range(world)]
        dist.all_gather(parts, flat)
        if rank == 0:
            phys = np.concatenate([p.view(torch.complex128).numpy() for p in parts])
            got = unpermute(phys, perm, n)
            out[rank] = float(np.max(np.abs(got - O.run_circuit(n, ops).a)))
        else:
            out[rank] = "ok"
    except Exception as e:  # the partner left: its exchange cannot complete
        out[rank] = "error: " + type(e).__name__
        return
    dist.destroy_process_group()


def _spawn(world, n, seed, leave_after=None, timeout=180):
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, seed, leave_after, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=timeout)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.exitcode is None:
            p.kill()
    return dict(out), codes


@pytest.mark.parametrize("world,n", [(2, 9), (4, 10)])
def test_gloo_ranks_exchange_halves_and_match_the_oracle(world, n):
    out, codes = _spawn(world, n, 900 + world)
    assert codes == [0] * world, (codes, out)
    assert isinstance(out[0], float) and out[0] <= 1e-12, out
    assert all(out[r] == "ok" for r in range(1, world)), out


def test_rank_leaving_between_steps_is_detected():
    """Rank 1 exits before its second exchange; rank 0's next exchange with
    it fails (connection closed or the group's timeout) instead of hanging,
    and rank 0 ends normally."""
    out, codes = _spawn(2, 9, 905, leave_after=1, timeout=120)
    assert out.get(1) == "left"
    assert str(out.get(0, "")).startswith("error"), out
    assert codes[0] == 0
