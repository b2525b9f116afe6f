"""Seeded workload generator: PRNG test vectors, layering rules, stream hashes."""
from collections import Counter

from paper_1802_08032_b300 import circuits as C


def test_splitmix64_published_vectors():
    # Outputs of the SplitMix64 reference generator for seeds 1234567 and 0.
    r = C.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]
    r = C.SplitMix64(0)
    assert [r.next_u64() for _ in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_layering_alternate():
    n, d = 30, 40
    ops = C.random_circuit(n, d, 8032, extras=True)
    assert [o.kind for o in ops[:n]] == ["H"] * n
    cnt = Counter(o.kind for o in ops)
    # CZ: 15 on odd layers (offset 0), 14 on even layers (offset 1)
    assert cnt["CZ"] == 20 * 15 + 19 * 14
    assert cnt["SX"] + cnt["SY"] + cnt["T"] == 39 * 15
    assert cnt["COMPACT"] == cnt["MCPF"] == 39
    assert len(ops) == 30 + 39 * 15 + 566 + 78
    for o in ops:
        if o.kind == "CZ":
            a, b = o.targets
            assert b == a + 1
        if o.kind == "MCPF":
            assert len(set(o.controls)) == 3
        if o.kind == "COMPACT":
            ar, ai, br, bi = o.params
            assert abs(ar * ar + ai * ai + br * br + bi * bi - 1) < 1e-15


def test_free_layering_skips_cz_qubits():
    ops = C.random_circuit(7, 5, 1, layering="free")
    layer_ops = ops[7:]
    i = 0
    for layer in range(1, 5):
        ncz = len(range((layer - 1) % 2, 6, 2))
        czs = layer_ops[i:i + ncz]
        busy = {q for o in czs for q in o.targets}
        i += ncz
        nfree = 7 - len(busy)
        singles = layer_ops[i:i + nfree]
        assert {o.targets[0] for o in singles} == set(range(7)) - busy
        i += nfree


def test_noise_follows_every_gate_qubit():
    ops = C.random_density_circuit(5, 4, 14, 0.01, 0.005)
    for k, o in enumerate(ops):
        if o.kind in C.CHANNELS:
            continue
        after = ops[k + 1:k + 1 + 2 * len(o.qubits())]
        assert [a.kind for a in after] == ["DEPHASE", "DEPOL"] * len(o.qubits())
        assert [a.targets[0] for a in after[::2]] == list(o.qubits())


def test_stream_hashes_are_stable():
    assert C.stream_hash(C.workload_12q()) == \
        "9524d95e8812b12324d2cde479b26991640b04e87b4efbfe131d65c719bd730e"
    assert C.stream_hash(C.workload_30q()) == \
        "722dac9b77ec993e95356572c1005e96510cc9e9a8ddb70213873ea0423a3b5c"
    assert C.stream_hash(C.workload_dm14()) == \
        "84b21a50638e263241b02f79c9ab4556d8ada8b1a185de8f57a1e637b9b75128"


def test_sample_indices():
    idx = C.sample_indices(20, 100, 5)
    assert len(idx) == 100 and idx[0] == 0 and idx[-1] == (1 << 20) - 1
    assert idx == sorted(set(idx))
