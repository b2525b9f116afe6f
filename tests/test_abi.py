"""The C-ABI library loads and exports every function include/qsim.h
declares; without a GPU it fails loudly instead of falling back (CPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?(?:int|char|void|double)\s*\*?\s*(\w+)\s*\(",
                            src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1802_08032_b300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_paper_api():
    names = set(declared_functions())
    for n in ["createQuESTEnv", "syncQuESTEnv", "createQureg", "createDensityQureg",
              "initZeroState", "hadamard", "compactUnitary", "unitary", "controlledNot",
              "controlledUnitary", "multiControlledPhaseFlip", "mixDephasing",
              "mixDepolarising", "calcTotalProb", "calcProbOfOutcome", "collapseToOutcome"]:
        assert n in names, n


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    from paper_1802_08032_b300 import qsim
    known = set(qsim.SIGNATURES) | set(qsim.EXTRA_SIGNATURES) | {"qsLastError"}
    assert set(declared_functions()) <= known
    for n in declared_functions():
        if n != "qsLastError":
            assert callable(getattr(qsim, n)), n


def test_no_gpu_means_loud_failure(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1802_08032_b300 import qsim
    with pytest.raises(qsim.QSimError) as e:
        qsim.createQuESTEnv()
    assert e.value.name == "QS_E_CUDA"


def test_status_codes_match_header():
    from paper_1802_08032_b300 import qsim
    src = open(os.path.join(ROOT, "include", "qsim.h")).read()
    for code, name in qsim.ERRORS.items():
        if name == "QS_OK":
            continue
        assert re.search(rf"{name}\s*=\s*{code}\b", src), name
    for name, code in qsim.OP_CODES.items():
        assert re.search(rf"QS_OP_\w+\s*=\s*{code}\b", src)


def test_matrix_marshalling_is_the_complex_layout():
    """Multi-target matrices go to the library as a pointer into contiguous
    complex128 (re, im per entry: the layout of Complex), row-major, sized
    4^m for m targets; other sizes are refused before the call."""
    import numpy as np
    from paper_1802_08032_b300 import qsim as Q
    u = (np.arange(16) + 1j * (100 + np.arange(16))).reshape(4, 4)
    a, p = Q._cmatrix(u, 2)
    for e in range(16):
        assert (p[e].re, p[e].im) == (u.reshape(-1)[e].real, u.reshape(-1)[e].imag)
    a, p = Q._cmatrix(u.T, 2)  # a transposed view is copied into row-major order
    assert (p[1].re, p[1].im) == (u[1, 0].real, u[1, 0].imag)
    for m in (1, 3):
        with pytest.raises(ValueError):
            Q._cmatrix(u, m)
