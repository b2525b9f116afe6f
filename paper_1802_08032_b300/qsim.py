"""Python binding of the C-ABI library libqsim.so (declared in include/qsim.h).

Argument marshalling only: every call goes straight to the library of the
same name, and every step of the simulation runs in its CUDA kernels.  There
is no CPU fallback: importing this module raises when libqsim.so is missing,
and the library itself needs a CUDA device.

Python-level differences from the C signatures: outputs are returned
instead of written through pointers, a failed call raises QSimError
(code, message) instead of returning a status, and Complex / matrix
arguments accept Python complex numbers and 2x2 nested sequences.
"""
from __future__ import annotations

import atexit
import ctypes
import os
from typing import Iterable, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqsim.so")

QS_C64, QS_C128 = 64, 128
ERRORS = {
    0: "QS_OK", -1: "QS_E_QUBIT", -2: "QS_E_DUP", -3: "QS_E_UNITARY", -4: "QS_E_PROB",
    -5: "QS_E_NOT_DENSITY", -6: "QS_E_ZERO_PROB", -7: "QS_E_NOMEM", -8: "QS_E_HANDLE",
    -9: "QS_E_CUDA", -10: "QS_E_TIMEOUT", -11: "QS_E_ARG", -12: "QS_E_BUSY",
}
OP_CODES = {"H": 1, "X": 2, "SX": 3, "SY": 4, "T": 5, "PHASE": 6, "COMPACT": 7,
            "UNITARY": 8, "CNOT": 9, "CUNITARY": 10, "CZ": 11, "MCPF": 12,
            "DEPHASE": 13, "DEPOL": 14}
MAX_OP_CONTROLS = 8


class QSimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


class Complex(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class ComplexMatrix2(ctypes.Structure):
    _fields_ = [("m", (Complex * 2) * 2)]


class ComplexMatrix4(ctypes.Structure):
    _fields_ = [("m", (Complex * 4) * 4)]


class QuESTEnv(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64)]


class Qureg(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64)]


class QSOp(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("target", ctypes.c_int32),
                ("target2", ctypes.c_int32), ("numControls", ctypes.c_int32),
                ("controls", ctypes.c_int32 * MAX_OP_CONTROLS),
                ("params", ctypes.c_double * 8)]


class QSBatch(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64)]


class QSServer(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64)]


class QSPartReg(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64)]


class QSPartStep(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("op", ctypes.c_int32), ("globalPos", ctypes.c_int32),
                ("localPos", ctypes.c_int32)]


class QSRequest(ctypes.Structure):
    _fields_ = [("isDensity", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("numQubits", ctypes.c_int32), ("measureQubit", ctypes.c_int32),
                ("ops", ctypes.c_void_p), ("numOps", ctypes.c_int64),
                ("outAmps", ctypes.c_void_p), ("outCount", ctypes.c_int64)]


class QSResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("totalProb", ctypes.c_double), ("probOutcome0", ctypes.c_double),
                ("queuedUs", ctypes.c_double), ("latencyUs", ctypes.c_double)]


class QSKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("flops", ctypes.c_double), ("alu_ops", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_P = ctypes.POINTER
_I, _I64, _D, _VP = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
# name -> argtypes (every function returns int status, except qsLastError)
SIGNATURES = {
    "createQuESTEnv": [_P(QuESTEnv)],
    "qsJitShutdown": [],
    "destroyQuESTEnv": [QuESTEnv],
    "syncQuESTEnv": [QuESTEnv],
    "qsDiagBoundedWait": [QuESTEnv, ctypes.c_int],
    "setEnvOption": [QuESTEnv, ctypes.c_char_p, _I64],
    "getEnvOption": [QuESTEnv, ctypes.c_char_p, _P(_I64)],
    "setAllocator": [QuESTEnv, ALLOC_FN, RELEASE_FN, _VP],
    "setStream": [QuESTEnv, _VP],
    "createQureg": [_I, _I, QuESTEnv, _P(Qureg)],
    "createDensityQureg": [_I, _I, QuESTEnv, _P(Qureg)],
    "destroyQureg": [Qureg],
    "initZeroState": [Qureg],
    "initPlusState": [Qureg],
    "copyStateToHost": [Qureg, _VP, _I64, _I64],
    "setAmps": [Qureg, _VP, _I64, _I64],
    "getNumQubits": [Qureg, _P(_I)],
    "getNumAmps": [Qureg, _P(_I64)],
    "getQuregInfo": [Qureg, _P(_I), _P(_I), _P(_I), _P(_VP)],
    "hadamard": [Qureg, _I],
    "pauliX": [Qureg, _I],
    "sqrtX": [Qureg, _I],
    "sqrtY": [Qureg, _I],
    "tGate": [Qureg, _I],
    "phaseShift": [Qureg, _I, _D],
    "compactUnitary": [Qureg, _I, Complex, Complex],
    "unitary": [Qureg, _I, ComplexMatrix2],
    "controlledNot": [Qureg, _I, _I],
    "controlledUnitary": [Qureg, _I, _I, ComplexMatrix2],
    "multiControlledUnitary": [Qureg, _P(_I), _I, _I, ComplexMatrix2],
    "controlledPhaseFlip": [Qureg, _I, _I],
    "multiQubitUnitary": [Qureg, _P(_I), _I, _P(Complex)],
    "multiControlledMultiQubitUnitary": [Qureg, _P(_I), _I, _P(_I), _I, _P(Complex)],
    "twoQubitUnitary": [Qureg, _I, _I, ComplexMatrix4],
    "multiControlledPhaseFlip": [Qureg, _P(_I), _I],
    "mixDephasing": [Qureg, _I, _D],
    "mixDepolarising": [Qureg, _I, _D],
    "calcTotalProb": [Qureg, _P(_D)],
    "calcProbOfOutcome": [Qureg, _I, _I, _P(_D)],
    "collapseToOutcome": [Qureg, _I, _I, _P(_D)],
    "calcPurity": [Qureg, _P(_D)],
    "calcInnerProduct": [Qureg, Qureg, _P(Complex)],
    "calcFidelity": [Qureg, Qureg, _P(_D)],
    "applyCircuit": [Qureg, _P(QSOp), _I64],
    "getKernelStats": [QuESTEnv, _P(QSKernelStat), _I, _P(_I)],
    "resetKernelStats": [QuESTEnv],
}
EXTRA_SIGNATURES: dict = {
    "calcTotalProbNoAlloc": [_VP, _I, _I64, _VP, _VP],
    "createBatch": [QuESTEnv, _P(Qureg), _I, _I, _P(QSBatch)],
    "runBatch": [QSBatch],
    "getBatchNorms": [QSBatch, _P(_D)],
    "getBatchInfo": [QSBatch, _P(_I), _P(_I64), _P(_I), _P(_D), _P(_D)],
    "tuneBatch": [QSBatch, _P(_I), _I, _I, _P(_I)],
    "tuneBatchJoint": [QSBatch, _P(_I), _I, _P(_I), _I, _I, _P(_I), _P(_I)],
    "destroyBatch": [QSBatch],
    "serveCreate": [QuESTEnv, _I, _I64, _I, _P(QSServer)],
    "serveSubmit": [QSServer, _P(QSRequest), _P(_I64)],
    "servePoll": [QSServer, _I64, _P(QSResult), _I64],
    "serveSetOption": [QSServer, ctypes.c_char_p, _I64],
    "serveGetOption": [QSServer, ctypes.c_char_p, _P(_I64)],
    "serveDestroy": [QSServer],
    "createPartitionedQureg": [_I, _I, _I, QuESTEnv, _P(QSPartReg)],
    "destroyPartitionedQureg": [QSPartReg],
    "partApplyCircuit": [QSPartReg, _P(QSOp), _I64],
    "partCalcTotalProb": [QSPartReg, _P(_D)],
    "partCalcProbOfOutcome": [QSPartReg, _I, _I, _P(_D)],
    "partCopyStateToHost": [QSPartReg, _VP],
    "partGetInfo": [QSPartReg, _P(_I), _P(_I), _P(_I), _P(_I64), _P(_D)],
    "partPlanSchedule": [_I, _I, _P(QSOp), _I64, _P(QSPartStep), _I64, _P(_I64), _P(_I)],
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library {LIB_PATH} is not built "
                          "(run paper_1802_08032_b300.build.build()); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    lib.qsLastError.restype = ctypes.c_char_p
    lib.qsLastError.argtypes = []
    for name, args in {**SIGNATURES, **EXTRA_SIGNATURES}.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    return lib


LIB = _load()


def qsJitShutdown():
    """Waits for background kernel compiles in flight and stops the compile
    threads (runs at interpreter exit, before the process tears down)."""
    _check(LIB.qsJitShutdown())


atexit.register(qsJitShutdown)


def _check(code: int):
    if code != 0:
        raise QSimError(code, LIB.qsLastError().decode(errors="replace"))


def _cplx(z) -> Complex:
    z = complex(z)
    return Complex(z.real, z.imag)


def _mat(u) -> ComplexMatrix2:
    m = ComplexMatrix2()
    for r in range(2):
        for c in range(2):
            z = complex(u[r][c])
            m.m[r][c] = Complex(z.real, z.imag)
    return m


def _ints(xs: Sequence[int]):
    arr = (ctypes.c_int * max(1, len(xs)))(*[int(x) for x in xs])
    return arr, len(xs)


# ------------------------------------------------------------ environment
def createQuESTEnv() -> QuESTEnv:
    e = QuESTEnv()
    _check(LIB.createQuESTEnv(ctypes.byref(e)))
    return e


def destroyQuESTEnv(env: QuESTEnv):
    _check(LIB.destroyQuESTEnv(env))


def syncQuESTEnv(env: QuESTEnv):
    _check(LIB.syncQuESTEnv(env))


def qsDiagBoundedWait(env: QuESTEnv, timeout_us: int):
    _check(LIB.qsDiagBoundedWait(env, int(timeout_us)))


def setEnvOption(env: QuESTEnv, key: str, value: int):
    _check(LIB.setEnvOption(env, key.encode(), int(value)))


def getEnvOption(env: QuESTEnv, key: str) -> int:
    v = ctypes.c_int64()
    _check(LIB.getEnvOption(env, key.encode(), ctypes.byref(v)))
    return v.value


_ALLOCATORS = {}


def setAllocator(env: QuESTEnv, alloc, release, ctx=None):
    """alloc(bytes) -> int device pointer (0 on failure); release(ptr)."""
    if alloc is None:
        _check(LIB.setAllocator(env, ALLOC_FN(), RELEASE_FN(), None))
        _ALLOCATORS.pop(env.id, None)
        return
    a = ALLOC_FN(lambda n, _ctx: alloc(n) or None)
    r = RELEASE_FN(lambda p, _ctx: release(p))
    _ALLOCATORS[env.id] = (a, r)        # keep the callbacks alive
    _check(LIB.setAllocator(env, a, r, None))


def use_torch_allocator(env: QuESTEnv):
    """Register memory from PyTorch's caching allocator on the current device."""
    import torch

    def alloc(n):
        return torch.cuda.caching_allocator_alloc(int(n))

    def release(p):
        torch.cuda.caching_allocator_delete(p)

    setAllocator(env, alloc, release)


def setStream(env: QuESTEnv, stream):
    """stream: a cudaStream_t as int, a torch.cuda.Stream, or None."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(LIB.setStream(env, ctypes.c_void_p(stream) if stream else None))


# -------------------------------------------------------------- registers
def createQureg(numQubits: int, precision: int, env: QuESTEnv) -> Qureg:
    q = Qureg()
    _check(LIB.createQureg(numQubits, precision, env, ctypes.byref(q)))
    return q


def createDensityQureg(numQubits: int, precision: int, env: QuESTEnv) -> Qureg:
    q = Qureg()
    _check(LIB.createDensityQureg(numQubits, precision, env, ctypes.byref(q)))
    return q


def destroyQureg(q: Qureg):
    _check(LIB.destroyQureg(q))


def initZeroState(q: Qureg):
    _check(LIB.initZeroState(q))


def initPlusState(q: Qureg):
    _check(LIB.initPlusState(q))


def copyStateToHost(q: Qureg, start: int = 0, count: int | None = None, out=None):
    """Returns a numpy complex128 array of `count` amplitudes from `start`."""
    import numpy as np
    if count is None:
        count = getNumAmps(q) - start
    if out is None:
        out = np.empty(count, dtype=np.complex128)
    assert out.dtype == np.complex128 and out.flags["C_CONTIGUOUS"] and out.size >= count
    _check(LIB.copyStateToHost(q, out.ctypes.data if count else None, int(start), int(count)))
    return out


def setAmps(q: Qureg, amps, start: int = 0):
    import numpy as np
    a = np.ascontiguousarray(amps, dtype=np.complex128)
    _check(LIB.setAmps(q, a.ctypes.data if a.size else None, int(start), int(a.size)))


def getNumQubits(q: Qureg) -> int:
    v = ctypes.c_int()
    _check(LIB.getNumQubits(q, ctypes.byref(v)))
    return v.value


def getNumAmps(q: Qureg) -> int:
    v = ctypes.c_int64()
    _check(LIB.getNumAmps(q, ctypes.byref(v)))
    return v.value


def getQuregInfo(q: Qureg):
    n, d, p, ptr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_void_p()
    _check(LIB.getQuregInfo(q, ctypes.byref(n), ctypes.byref(d), ctypes.byref(p), ctypes.byref(ptr)))
    return {"numQubits": n.value, "isDensity": bool(d.value), "precision": p.value,
            "devicePtr": ptr.value}


# ------------------------------------------------------------------ gates
def hadamard(q, t): _check(LIB.hadamard(q, t))
def pauliX(q, t): _check(LIB.pauliX(q, t))
def sqrtX(q, t): _check(LIB.sqrtX(q, t))
def sqrtY(q, t): _check(LIB.sqrtY(q, t))
def tGate(q, t): _check(LIB.tGate(q, t))
def phaseShift(q, t, angle): _check(LIB.phaseShift(q, t, float(angle)))


def compactUnitary(q, t, alpha, beta):
    _check(LIB.compactUnitary(q, t, _cplx(alpha), _cplx(beta)))


def unitary(q, t, u):
    _check(LIB.unitary(q, t, _mat(u)))


def controlledNot(q, c, t): _check(LIB.controlledNot(q, c, t))


def controlledUnitary(q, c, t, u):
    _check(LIB.controlledUnitary(q, c, t, _mat(u)))


def multiControlledUnitary(q, controls: Sequence[int], t, u):
    arr, n = _ints(controls)
    _check(LIB.multiControlledUnitary(q, arr, n, t, _mat(u)))


def controlledPhaseFlip(q, a, b): _check(LIB.controlledPhaseFlip(q, a, b))


def _cmatrix(u, m: int):
    """A 2^m x 2^m matrix as contiguous complex128 (the layout of Complex,
    re then im) and a pointer into it, without a copy when u already is one;
    the caller keeps the array alive for the call."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(u, dtype=np.complex128).reshape(-1))
    if m < 0 or a.size != 1 << (2 * m):
        raise ValueError(f"matrix has {a.size} entries; {m} targets need {1 << (2 * max(m, 0))}")
    return a, a.ctypes.data_as(ctypes.POINTER(Complex))


def multiQubitUnitary(q, targets: Sequence[int], u):
    """u: 2^m x 2^m unitary (bit k of its index is targets[k])."""
    t, n = _ints(targets)
    a, p = _cmatrix(u, n)
    _check(LIB.multiQubitUnitary(q, t, n, p))


def multiControlledMultiQubitUnitary(q, controls: Sequence[int], targets: Sequence[int], u):
    c, nc = _ints(controls)
    t, nt = _ints(targets)
    a, p = _cmatrix(u, nt)
    _check(LIB.multiControlledMultiQubitUnitary(q, c, nc, t, nt, p))


def twoQubitUnitary(q, t1, t2, u):
    m = ComplexMatrix4()
    for r in range(4):
        for c in range(4):
            z = complex(u[r][c])
            m.m[r][c] = Complex(z.real, z.imag)
    _check(LIB.twoQubitUnitary(q, t1, t2, m))


def multiControlledPhaseFlip(q, controls: Sequence[int]):
    arr, n = _ints(controls)
    _check(LIB.multiControlledPhaseFlip(q, arr, n))


def mixDephasing(q, t, p): _check(LIB.mixDephasing(q, t, float(p)))
def mixDepolarising(q, t, p): _check(LIB.mixDepolarising(q, t, float(p)))


# ------------------------------------------------------------- reductions
def calcTotalProb(q) -> float:
    v = ctypes.c_double()
    _check(LIB.calcTotalProb(q, ctypes.byref(v)))
    return v.value


def calcProbOfOutcome(q, qubit, outcome) -> float:
    v = ctypes.c_double()
    _check(LIB.calcProbOfOutcome(q, qubit, outcome, ctypes.byref(v)))
    return v.value


def collapseToOutcome(q, qubit, outcome) -> float:
    v = ctypes.c_double()
    _check(LIB.collapseToOutcome(q, qubit, outcome, ctypes.byref(v)))
    return v.value


def calcInnerProduct(bra, ket) -> complex:
    out = Complex()
    _check(LIB.calcInnerProduct(bra, ket, ctypes.byref(out)))
    return complex(out.re, out.im)


def calcFidelity(a, b) -> float:
    out = ctypes.c_double()
    _check(LIB.calcFidelity(a, b, ctypes.byref(out)))
    return out.value


def calcPurity(q) -> float:
    v = ctypes.c_double()
    _check(LIB.calcPurity(q, ctypes.byref(v)))
    return v.value


# ------------------------------------------------------------- bulk calls
def to_qsops(ops: Iterable) -> ctypes.Array:
    """Gate list (circuits.Op tuples) -> contiguous QSOp array."""
    ops = list(ops)
    arr = (QSOp * max(1, len(ops)))()
    for i, op in enumerate(ops):
        o = arr[i]
        o.kind = OP_CODES[op.kind]
        tg = tuple(op.targets)
        o.target = tg[0] if tg else -1
        o.target2 = tg[1] if len(tg) > 1 else -1
        ctr = tuple(op.controls)
        if len(ctr) > MAX_OP_CONTROLS:
            raise ValueError("too many controls for one QSOp")
        o.numControls = len(ctr)
        for k, c in enumerate(ctr):
            o.controls[k] = c
        for k, p in enumerate(op.params):
            o.params[k] = float(p)
    return arr, len(ops)


def applyCircuit(q, ops):
    """ops: a QSOp array from to_qsops, or a gate list."""
    if isinstance(ops, tuple) and len(ops) == 2 and isinstance(ops[1], int):
        arr, n = ops
    else:
        arr, n = to_qsops(ops)
    _check(LIB.applyCircuit(q, arr, n))


# ------------------------------------------------------------ kernel stats
def getKernelStats(env) -> list:
    """[{name, launches, total_ms, bytes, flops}] per kernel class."""
    cnt = ctypes.c_int()
    _check(LIB.getKernelStats(env, None, 0, ctypes.byref(cnt)))
    arr = (QSKernelStat * max(1, cnt.value))()
    _check(LIB.getKernelStats(env, arr, cnt.value, ctypes.byref(cnt)))
    return [{"name": a.name.decode(), "launches": a.launches, "total_ms": a.total_ms,
             "bytes": a.bytes, "flops": a.flops, "alu_ops": a.alu_ops} for a in arr[:cnt.value]]


def resetKernelStats(env):
    _check(LIB.resetKernelStats(env))


# ------------------------------------------------- allocation-free norm
def calcTotalProbNoAlloc(amps_ptr: int, precision: int, num_amps: int, out_ptr: int,
                         stream=None):
    """Queues sum |amps|^2 (FP64) into the device double at out_ptr, with no
    device allocation (for callers that cannot allocate).  amps_ptr and
    out_ptr are device addresses owned by the caller; stream is a cudaStream_t
    as int, a torch.cuda.Stream, or None (legacy default stream).  The call
    does not wait for the result."""
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    _check(LIB.calcTotalProbNoAlloc(ctypes.c_void_p(amps_ptr), int(precision), int(num_amps),
                                    ctypes.c_void_p(out_ptr),
                                    ctypes.c_void_p(stream) if stream else None))


# ------------------------------------------------------------- batches
def createBatch(env, regs, tileQubits: int = 0) -> QSBatch:
    arr = (Qureg * len(regs))(*[Qureg(r.id) for r in regs])
    b = QSBatch()
    _check(LIB.createBatch(env, arr, len(regs), int(tileQubits), ctypes.byref(b)))
    b.count = len(regs)
    return b


def runBatch(b):
    _check(LIB.runBatch(b))


def getBatchNorms(b, count=None):
    import numpy as np
    n = count if count is not None else b.count
    out = np.empty(n, dtype=np.float64)
    _check(LIB.getBatchNorms(b, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def getBatchInfo(b) -> dict:
    k, p, w, by, fl = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    _check(LIB.getBatchInfo(b, ctypes.byref(k), ctypes.byref(p), ctypes.byref(w), ctypes.byref(by),
                            ctypes.byref(fl)))
    return {"tileQubits": k.value, "passes": p.value, "waves": w.value, "bytes": by.value,
            "flops": fl.value}


def tuneBatch(b, candidates, replays: int = 2) -> int:
    arr, n = _ints(candidates)
    c = ctypes.c_int()
    _check(LIB.tuneBatch(b, arr, n, int(replays), ctypes.byref(c)))
    return c.value


def tuneBatchJoint(b, tiles, depths, replays: int = 1):
    """Times every (tile size, fusion depth) pair; returns the fastest."""
    ta, da = _ints(tiles), _ints(depths)
    ck, cd = ctypes.c_int(), ctypes.c_int()
    _check(LIB.tuneBatchJoint(b, ta[0], ta[1], da[0], da[1], int(replays), ctypes.byref(ck), ctypes.byref(cd)))
    return ck.value, cd.value


def destroyBatch(b):
    _check(LIB.destroyBatch(b))


# ------------------------------------------------------------- serving
def serveCreate(env, slots: int, budgetBytes: int, fusion: int = 1) -> QSServer:
    s = QSServer()
    _check(LIB.serveCreate(env, int(slots), int(budgetBytes), int(fusion), ctypes.byref(s)))
    s._keep = {}
    return s


def serveSubmit(server, ops, numQubits: int, precision: int = QS_C64, isDensity: bool = False,
                measureQubit: int = 0, outAmps=None) -> int:
    """Queues one circuit; ops is a gate list or a to_qsops() pair.  outAmps:
    optional numpy complex128 array that receives the first outAmps.size
    final amplitudes (kept alive until servePoll returns the result)."""
    arr, n = ops if (isinstance(ops, tuple) and len(ops) == 2 and isinstance(ops[1], int)) \
        else to_qsops(ops)
    r = QSRequest(int(bool(isDensity)), int(precision), int(numQubits), int(measureQubit),
                  ctypes.cast(arr, ctypes.c_void_p), int(n),
                  outAmps.ctypes.data if outAmps is not None else None,
                  int(outAmps.size) if outAmps is not None else 0)
    t = ctypes.c_int64()
    _check(LIB.serveSubmit(server, ctypes.byref(r), ctypes.byref(t)))
    if outAmps is not None:
        server._keep[t.value] = outAmps
    return t.value


def servePoll(server, ticket: int, timeoutUs: int = 60_000_000) -> dict:
    res = QSResult()
    _check(LIB.servePoll(server, int(ticket), ctypes.byref(res), int(timeoutUs)))
    server._keep.pop(ticket, None)
    return {"status": res.status, "slot": res.slot, "totalProb": res.totalProb,
            "probOutcome0": res.probOutcome0, "queuedUs": res.queuedUs,
            "latencyUs": res.latencyUs}


def serveSetOption(server, key: str, value: int):
    _check(LIB.serveSetOption(server, key.encode(), int(value)))


def serveGetOption(server, key: str) -> int:
    v = ctypes.c_int64()
    _check(LIB.serveGetOption(server, key.encode(), ctypes.byref(v)))
    return v.value


def serveDestroy(server):
    _check(LIB.serveDestroy(server))


# ------------------------------------------------ partitioned registers
def createPartitionedQureg(numQubits: int, globalQubits: int, precision: int, env) -> QSPartReg:
    r = QSPartReg()
    _check(LIB.createPartitionedQureg(int(numQubits), int(globalQubits), int(precision), env, ctypes.byref(r)))
    return r


def destroyPartitionedQureg(r):
    _check(LIB.destroyPartitionedQureg(r))


def partApplyCircuit(r, ops):
    arr, n = ops if (isinstance(ops, tuple) and len(ops) == 2 and isinstance(ops[1], int)) else to_qsops(ops)
    _check(LIB.partApplyCircuit(r, arr, n))


def partCalcTotalProb(r) -> float:
    out = ctypes.c_double()
    _check(LIB.partCalcTotalProb(r, ctypes.byref(out)))
    return out.value


def partCalcProbOfOutcome(r, qubit: int, outcome: int) -> float:
    out = ctypes.c_double()
    _check(LIB.partCalcProbOfOutcome(r, int(qubit), int(outcome), ctypes.byref(out)))
    return out.value


def partCopyStateToHost(r):
    import numpy as np
    info = partGetInfo(r)
    out = np.empty(1 << info["numQubits"], dtype=np.complex128)
    _check(LIB.partCopyStateToHost(r, out.ctypes.data))
    return out


def partGetInfo(r) -> dict:
    n, k = ctypes.c_int(), ctypes.c_int()
    _check(LIB.partGetInfo(r, ctypes.byref(n), ctypes.byref(k), None, None, None))
    perm = (ctypes.c_int * n.value)()
    sw, ex = ctypes.c_int64(), ctypes.c_double()
    _check(LIB.partGetInfo(r, None, None, perm, ctypes.byref(sw), ctypes.byref(ex)))
    return {"numQubits": n.value, "globalQubits": k.value, "perm": list(perm), "swaps": sw.value,
            "exchangedBytes": ex.value}


def partPlanSchedule(numQubits: int, globalQubits: int, ops):
    """Host-only schedule: ([(kind, op, globalPos, localPos)], final qubit map)."""
    arr, n = ops if (isinstance(ops, tuple) and len(ops) == 2 and isinstance(ops[1], int)) else to_qsops(ops)
    cnt = ctypes.c_int64()
    perm = (ctypes.c_int * numQubits)()
    _check(LIB.partPlanSchedule(int(numQubits), int(globalQubits), arr, n, None, 0, ctypes.byref(cnt), perm))
    steps = (QSPartStep * max(1, cnt.value))()
    _check(LIB.partPlanSchedule(int(numQubits), int(globalQubits), arr, n, steps, cnt.value, ctypes.byref(cnt),
                                perm))
    return [(s.kind, s.op, s.globalPos, s.localPos) for s in steps[:cnt.value]], list(perm)
