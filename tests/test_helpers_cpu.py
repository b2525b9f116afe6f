"""CPU checks of test helpers that GPU tests rely on (no GPU needed)."""
import numpy as np

from oracle import oracle as O
from paper_1802_08032_b300 import circuits as C
from gpu_helpers import inverse


def test_mirror_helper_returns_zero_state():
    """C followed by inverse(C) is the identity on the oracle: the closed form
    the 33-qubit mirror test relies on (a wrong inverse of any gate kind of
    the workload would leave a state other than |0...0>)."""
    for seed in (77, 78, 79):
        ops = C.random_circuit(5, 12, seed, extras=True)
        assert {o.kind for o in ops} >= {C.H, C.CZ, C.MCPF, C.T_GATE, C.SQRT_X, C.SQRT_Y, C.COMPACT}
        st = O.run_circuit(5, ops + inverse(ops))
        want = np.zeros(32, complex)
        want[0] = 1
        assert np.max(np.abs(st.a - want)) <= 1e-13
        # and C alone is far from it (the check is not vacuous)
        assert abs(O.run_circuit(5, ops).a[0]) < 0.9
