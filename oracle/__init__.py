"""CPU FP64 oracle for the matrix-valued biquaternion product (test infrastructure).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline / reference arm are the only callers.  The product path
(``paper_2609_02081_gb300``) never imports this package, and this package never
imports the product path; the two share only the seeded input generators in
``bq_inputs``.

Contents
--------
* ``oracle.c`` (compiled on first use with gcc): the component-wise
  64-real-product definition of C <- alpha op(A) op(B) + beta C
  (Sec. II A Eq. MatrixQMultiplication; Sec. III storage, op and scaling
  equations).  Wrapped here by :func:`bq_gemm` and :func:`apply_op`.
* ``isomorph.py``: the independent cross-check on the isomorphic complex
  2m x 2n representation (Sec. II A Eq. TRG-in-C, Sec. III M+/M- blocks and
  Eq. mapping-formulas), multiplied with numpy.
* ``ops.py``: the element-wise operations of Sec. III (complex scaling,
  addition, trace), the Hermiticity deviation, and the Hadamard block
  reduction of Sec. III C (Eq. hadamard_general_transform), in numpy; pinned
  in tests/test_oracle_ops_pins.py.

Parity pins: every function here is pinned in tests/test_oracle_pins.py to
values the paper and the mathematics fix (quaternion relations, the Pauli
isomorphism, brute force on the isomorph, associativity, the conjugation
identities, subalgebra reductions).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

OP_N, OP_T, OP_C, OP_H, OP_QC = 0, 1, 2, 3, 4
OP_NAMES = {"N": OP_N, "T": OP_T, "C": OP_C, "H": OP_H, "QC": OP_QC}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, dbl, ptr = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
            lib.oracle_apply_op.argtypes = [ctypes.c_int, i64, i64, ptr, ptr]
            lib.oracle_apply_op.restype = ctypes.c_int
            lib.oracle_bq_gemm_rows.argtypes = [i64, i64, i64, dbl, dbl, ptr, ptr, dbl, dbl,
                                                ptr, ptr, i64, ptr, ctypes.c_int]
            lib.oracle_bq_gemm_rows.restype = ctypes.c_int
            lib.oracle_max_threads.argtypes = []
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float64)


def _op_code(op) -> int:
    if isinstance(op, str):
        return OP_NAMES[op]
    return int(op)


def apply_op(op, X: np.ndarray) -> np.ndarray:
    """op(X) for an 8 x rows x cols biquaternion matrix (Sec. III op equations)."""
    X = _f64(X)
    if X.ndim != 3 or X.shape[0] != 8:
        raise ValueError("expected an 8 x rows x cols array")
    code = _op_code(op)
    rows, cols = X.shape[1], X.shape[2]
    shape = (8, cols, rows) if code in (OP_T, OP_H) else (8, rows, cols)
    Y = np.empty(shape, dtype=np.float64)
    if _load().oracle_apply_op(code, rows, cols, X.ctypes.data, Y.ctypes.data) != 0:
        raise ValueError(f"unknown op {op!r}")
    return Y


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def bq_gemm(A: np.ndarray, B: np.ndarray, opA="N", opB="N", alpha=1.0, beta=0.0,
            C: np.ndarray | None = None, rows=None, threads: int = 0) -> np.ndarray:
    """alpha * op(A) op(B) + beta * C with the component-wise 64-product definition.

    A, B, C are 8 x rows x cols float64 arrays (component-major, Sec. III
    Eq. biquat-repres).  ``rows`` selects output rows (default: all); the
    result then has shape 8 x len(rows) x n and C (if given) is the full
    8 x m x n matrix whose selected rows are read.  alpha and beta are complex
    scalars.  With beta == 0, C is not read.
    """
    Aop = apply_op(opA, A)
    Bop = apply_op(opB, B)
    m, k = Aop.shape[1], Aop.shape[2]
    if Bop.shape[1] != k:
        raise ValueError(f"inner dimensions differ: op(A) is {m}x{k}, op(B) is {Bop.shape[1]}x{Bop.shape[2]}")
    n = Bop.shape[2]
    row_idx = np.arange(m, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    alpha, beta = complex(alpha), complex(beta)
    C_in = None
    if beta != 0:
        if C is None:
            raise ValueError("beta != 0 needs C")
        C = _f64(C)
        if C.shape != (8, m, n):
            raise ValueError("C has the wrong shape")
        C_in = np.ascontiguousarray(C[:, row_idx, :])
    out = np.empty((8, row_idx.size, n), dtype=np.float64)
    rc = _load().oracle_bq_gemm_rows(
        m, n, k, alpha.real, alpha.imag, Aop.ctypes.data, Bop.ctypes.data,
        beta.real, beta.imag, None if C_in is None else C_in.ctypes.data,
        row_idx.ctypes.data, row_idx.size, out.ctypes.data, int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_bq_gemm_rows failed with {rc}")
    return out
