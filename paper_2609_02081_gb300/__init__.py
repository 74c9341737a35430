"""Python binding of libhmat (include/hmat.h): GB300 biquaternion matrix products.

The binding only marshals arguments: every step of the computation runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  There is
no CPU fallback; if the library cannot be built or loaded, :func:`lib` raises.

Matrices are torch float64 tensors of shape (8, rows, cols) on the GPU: the
eight real components [M1..M8] = [E_R, E_I, F_R, F_I, G_I, -G_R, H_I, -H_R] of
a biquaternion matrix (arXiv 2609.02081, Sec. III), each component row-major
(last stride 1); ``stride(1)`` is the leading dimension, ``stride(0)`` the
component stride.

    import paper_2609_02081_gb300 as hm
    with hm.Handle() as h:
        hm.hmat_bq_gemm(h, A, B, C, "N", "H", mode="split", tol=1e-12)   # C = A B^dagger
        hm.hmat_bq_gemm_grouped(h, [hm.make_desc(A1, B1, C1), hm.make_desc(A2, B2, C2)],
                                mode="split", tol=1e-12, use_graph=True)
        hm.hmat_bq_gemm_streamed(h, A_host, B_host, C_host, mode="split", tol=1e-12,
                                 budget=64 << 30)                        # pinned host operands
        hm.hmat_bq_add(h, A, B, C, alpha=1.0, beta=1j)                  # C = A + i B
        Z = hm.hmat_bq_to_complex(h, A)                                 # complex 2m x 2n image
        h.set_algorithm("standard")                                     # comparison algorithms
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

HMAT_OP_N, HMAT_OP_T, HMAT_OP_C, HMAT_OP_H, HMAT_OP_QC = 0, 1, 2, 3, 4
OPS = {"N": HMAT_OP_N, "T": HMAT_OP_T, "C": HMAT_OP_C, "H": HMAT_OP_H, "QC": HMAT_OP_QC}
HMAT_REAL, HMAT_COMPLEX, HMAT_TRS, HMAT_TRA, HMAT_BQ = 0x01, 0x11, 0x0F, 0xF0, 0xFF
HMAT_MODE_FP64, HMAT_MODE_SPLIT = 0, 1
HMAT_ALGO_BILINEAR, HMAT_ALGO_STANDARD, HMAT_ALGO_ISOMORPH = 0, 1, 2
ALGOS = {"bilinear": HMAT_ALGO_BILINEAR, "standard": HMAT_ALGO_STANDARD, "isomorph": HMAT_ALGO_ISOMORPH}
HMAT_CFORM_AUTO, HMAT_CFORM_GAUSS, HMAT_CFORM_FOUR_M = 0, 1, 2
CFORMS = {"auto": HMAT_CFORM_AUTO, "gauss": HMAT_CFORM_GAUSS, "four_m": HMAT_CFORM_FOUR_M}
HMAT_PLAN_INFO_FOUR_M = 3       # plan_info only: the split mode's four-multiplication form, two terms per product
MODES = {"fp64": HMAT_MODE_FP64, "split": HMAT_MODE_SPLIT}
KERNEL_IDS = {"fp64_bilinear": 0, "split_exponents": 1, "split_encode": 2, "split_residue_gemm": 3,
              "split_crt": 4, "beta_scale": 5, "iso_map_in": 6, "iso_map_out": 7, "add": 8, "to_complex": 9,
              "from_complex": 10, "trace": 11, "hermiticity": 12, "hadamard": 13, "fp64_splitk_reduce": 14}
STATUS = {0: "SUCCESS", 1: "INVALID_VALUE", 2: "UNSUPPORTED", 3: "MISALIGNED", 4: "WORKSPACE_TOO_SMALL",
          5: "CUDA_ERROR", 6: "DEVICE_TIMEOUT", 7: "NOT_INITIALIZED", 8: "TOLERANCE_UNREACHABLE", 9: "INTERNAL"}


class HmatError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: hmat status {status} ({STATUS.get(int(status), '?')})")


class hmat_gemm_desc(ctypes.Structure):
    _fields_ = [("opA", ctypes.c_int32), ("opB", ctypes.c_int32),
                ("flagsA", ctypes.c_uint32), ("flagsB", ctypes.c_uint32),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int64),
                ("alpha_re", ctypes.c_double), ("alpha_im", ctypes.c_double),
                ("beta_re", ctypes.c_double), ("beta_im", ctypes.c_double),
                ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("strideA", ctypes.c_int64),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("strideB", ctypes.c_int64),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64), ("strideC", ctypes.c_int64)]


_i32, _u32, _i64, _dbl, _ptr, _sz = (ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_size_t)
# name -> (restype, argtypes), mirroring include/hmat.h
SIGNATURES = {
    "hmat_version": (_i32, []),
    "hmat_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "hmat_last_cuda_error": (ctypes.c_char_p, []),
    "hmat_create": (ctypes.c_int, [ctypes.POINTER(_ptr)]),
    "hmat_destroy": (ctypes.c_int, [_ptr]),
    "hmat_workspace_size": (ctypes.c_int, [_ptr, _i32, ctypes.POINTER(hmat_gemm_desc), _i32, _dbl,
                                           ctypes.POINTER(_sz)]),
    "hmat_bq_gemm": (ctypes.c_int, [_ptr, _i32, _i32, _u32, _u32, _i64, _i64, _i64, _dbl, _dbl,
                                    _ptr, _i64, _i64, _ptr, _i64, _i64, _dbl, _dbl, _ptr, _i64, _i64,
                                    _i32, _dbl, _ptr, _sz, _ptr]),
    "hmat_bq_gemm_grouped": (ctypes.c_int, [_ptr, _i32, ctypes.POINTER(hmat_gemm_desc), _i32, _dbl, _ptr, _sz,
                                            _ptr, _i32]),
    "hmat_bq_gemm_grouped_modes": (ctypes.c_int, [_ptr, _i32, ctypes.POINTER(hmat_gemm_desc),
                                                  ctypes.POINTER(_i32), _dbl, _ptr, _sz, _ptr, _i32]),
    "hmat_workspace_size_modes": (ctypes.c_int, [_ptr, _i32, ctypes.POINTER(hmat_gemm_desc), ctypes.POINTER(_i32),
                                                 _dbl, ctypes.POINTER(_sz)]),
    "hmat_bq_gemm_split_noalloc": (ctypes.c_int, [_ptr, _i32, _i32, _u32, _u32, _i64, _i64, _i64, _dbl, _dbl,
                                                  _ptr, _i64, _i64, _ptr, _i64, _i64, _dbl, _dbl, _ptr, _i64, _i64,
                                                  _dbl, _ptr]),
    "hmat_split_noalloc_capacity": (_sz, []),
    "hmat_last_bad_index": (_i32, [_ptr]),
    "hmat_plan_info": (ctypes.c_int, [_i32, _i32, _i32, _u32, _u32, ctypes.POINTER(_i32), ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(_i32)]),
    "hmat_set_algorithm": (ctypes.c_int, [_ptr, _i32]),
    "hmat_set_complex_form": (ctypes.c_int, [_ptr, _i32]),
    "hmat_split_info": (ctypes.c_int, [_i64, _dbl, ctypes.POINTER(_i32), ctypes.c_void_p, ctypes.POINTER(_i32)]),
    "hmat_get_device_error": (ctypes.c_int, [_ptr, ctypes.POINTER(_u32)]),
    "hmat_set_tile_table": (ctypes.c_int, [_ptr, ctypes.c_void_p]),
    "hmat_set_tile_table_flags": (ctypes.c_int, [_ptr, _u32, _u32, ctypes.c_void_p]),
    "hmat_set_fp64_splitk_table": (ctypes.c_int, [_ptr, ctypes.c_void_p]),
    "hmat_debug_wait_selftest": (ctypes.c_int, [_ptr, _i64, _ptr]),
    "hmat_measure_fp64_peak": (ctypes.c_int, [_i32, _i64, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)]),
    "hmat_set_profiling": (ctypes.c_int, [_ptr, _i32]),
    "hmat_get_profile": (ctypes.c_int, [_ptr, _i32, ctypes.POINTER(_i64), ctypes.POINTER(_dbl)]),
    "hmat_reset_profile": (ctypes.c_int, [_ptr]),
    "hmat_streamed_plan": (ctypes.c_int, [_ptr, _i32, _i32, _u32, _u32, _i64, _i64, _i64, _i32, _dbl, _sz, _i32,
                                          _i32, _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                          ctypes.POINTER(_i64), ctypes.POINTER(_sz)]),
    "hmat_streamed_traffic": (ctypes.c_int, [_ptr, _i32, _i32, _u32, _u32, _i64, _i64, _i64, _i32, _dbl, _sz,
                                             _i32, _i32, _i32, _i32, ctypes.POINTER(_sz), ctypes.POINTER(_sz)]),
    "hmat_bq_gemm_streamed": (ctypes.c_int, [_ptr, _i32, _i32, _u32, _u32, _i64, _i64, _i64, _dbl, _dbl,
                                             _ptr, _i64, _i64, _ptr, _i64, _i64, _dbl, _dbl, _ptr, _i64, _i64,
                                             _i32, _dbl, _ptr, _sz, _ptr]),
    "hmat_bq_add": (ctypes.c_int, [_ptr, _i32, _i32, _u32, _u32, _i64, _i64, _dbl, _dbl, _ptr, _i64, _i64,
                                   _dbl, _dbl, _ptr, _i64, _i64, _ptr, _i64, _i64, _ptr]),
    "hmat_bq_scale": (ctypes.c_int, [_ptr, _i32, _u32, _i64, _i64, _dbl, _dbl, _ptr, _i64, _i64, _ptr, _i64, _i64,
                                     _ptr]),
    "hmat_bq_trace": (ctypes.c_int, [_ptr, _i32, _u32, _i64, _ptr, _i64, _i64, _ptr, _ptr]),
    "hmat_bq_to_complex": (ctypes.c_int, [_ptr, _i32, _u32, _i64, _i64, _ptr, _i64, _i64, _ptr, _i64, _ptr]),
    "hmat_complex_to_bq": (ctypes.c_int, [_ptr, _i64, _i64, _ptr, _i64, _ptr, _i64, _i64, _ptr]),
    "hmat_bq_hermiticity": (ctypes.c_int, [_ptr, _u32, _i64, _ptr, _i64, _i64, _ptr, _ptr]),
    "hmat_bq_hadamard_block": (ctypes.c_int, [_ptr, _u32, _i64, _dbl, _dbl, _ptr, _i64, _i64, _ptr, _i64, _ptr,
                                              _ptr]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """The loaded libhmat.so (built in-tree with nvcc on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"libhmat.so not found at {path}; run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        if status == 5:
            what = f"{what} [{lib().hmat_last_cuda_error().decode()}]"
        raise HmatError(status, what)


# ----------------------------------------------------------------------------- host-only queries
def plan_info(opA="N", opB="N", flagsA=HMAT_BQ, flagsB=HMAT_BQ, algo="bilinear"):
    """(n_products, U[P,8], V[P,8], W[8,P], strategy) of the product plan (hmat_plan_info);
    algo "four_m" lists the split mode's four-multiplication form as two terms per product."""
    L = lib()
    n = _i32()
    st = _i32()
    U = np.zeros((64, 8), dtype=np.int8)
    V = np.zeros((64, 8), dtype=np.int8)
    W = np.zeros((8, 64), dtype=np.float64)
    a = (HMAT_PLAN_INFO_FOUR_M if algo == "four_m" else ALGOS[algo]) if isinstance(algo, str) else int(algo)
    _check(L.hmat_plan_info(a, _op(opA), _op(opB), flagsA, flagsB, ctypes.byref(n), U.ctypes.data, V.ctypes.data,
                            W.ctypes.data, ctypes.byref(st)), "hmat_plan_info")
    P = n.value
    return P, U[:P].copy(), V[:P].copy(), W[:, :P].copy(), st.value


def split_info(k: int, tol: float = 0.0):
    """(moduli list, bits) that split mode uses for inner dimension k and tolerance tol."""
    L = lib()
    n = _i32()
    bits = _i32()
    mods = np.zeros(32, dtype=np.int32)
    _check(L.hmat_split_info(int(k), float(tol), ctypes.byref(n), mods.ctypes.data, ctypes.byref(bits)),
           "hmat_split_info")
    return [int(x) for x in mods[:n.value]], bits.value


FP64_PEAK_KINDS = {"dfma": 0, "dmma_m8n8k4": 1, "dmma_m16n8k4": 2}


def measure_fp64_peak(kind="dfma", iterations: int = 1 << 16):
    """(TFLOP/s, ms) of one FP64 probe launch on the current device (hmat_measure_fp64_peak)."""
    tf, ms = _dbl(), _dbl()
    _check(lib().hmat_measure_fp64_peak(FP64_PEAK_KINDS[kind], int(iterations), ctypes.byref(tf), ctypes.byref(ms)),
           "hmat_measure_fp64_peak")
    return tf.value, ms.value


def _op(op) -> int:
    return OPS[op] if isinstance(op, str) else int(op)


def _mode(mode) -> int:
    return MODES[mode] if isinstance(mode, str) else int(mode)


# ----------------------------------------------------------------------------- handle and calls
class Handle:
    """An hmat_handle bound to the current CUDA device."""

    def __init__(self):
        self._h = _ptr()
        _check(lib().hmat_create(ctypes.byref(self._h)), "hmat_create")

    @property
    def value(self):
        return self._h

    def close(self):
        if self._h:
            lib().hmat_destroy(self._h)
            self._h = _ptr()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- profiling / errors
    def set_profiling(self, on: bool):
        _check(lib().hmat_set_profiling(self._h, 1 if on else 0), "hmat_set_profiling")

    def profile(self, kernel: str):
        n = _i64()
        ms = _dbl()
        _check(lib().hmat_get_profile(self._h, KERNEL_IDS[kernel], ctypes.byref(n), ctypes.byref(ms)),
               "hmat_get_profile")
        return n.value, ms.value

    def reset_profile(self):
        _check(lib().hmat_reset_profile(self._h), "hmat_reset_profile")

    def set_algorithm(self, algo):
        """'bilinear' (default), 'standard' (component-wise, HMAT-standard) or 'isomorph' (CMAT)."""
        a = ALGOS[algo] if isinstance(algo, str) else int(algo)
        _check(lib().hmat_set_algorithm(self._h, a), "hmat_set_algorithm")

    def set_complex_form(self, form):
        """Complex-product form of split-mode full-biquaternion products: 'auto' (default: the
        four-multiplication form for k <= 512), 'gauss' (three real products, as in the paper)
        or 'four_m' (two real products over 2 k)."""
        f = CFORMS[form] if isinstance(form, str) else int(form)
        _check(lib().hmat_set_complex_form(self._h, f), "hmat_set_complex_form")

    def set_tile_table(self, table):
        """Install a 16 x 16 tile-width code table (None: built-in rule); see autotune.py."""
        if table is None:
            _check(lib().hmat_set_tile_table(self._h, None), "hmat_set_tile_table")
            return
        t = np.ascontiguousarray(table, dtype=np.int8).reshape(16, 16)
        _check(lib().hmat_set_tile_table(self._h, t.ctypes.data), "hmat_set_tile_table")

    def set_tile_table_flags(self, flagsA, flagsB, table):
        """Install a tile-width code table for products of one flag pair (None removes it)."""
        if table is None:
            _check(lib().hmat_set_tile_table_flags(self._h, int(flagsA), int(flagsB), None),
                   "hmat_set_tile_table_flags")
            return
        t = np.ascontiguousarray(table, dtype=np.int8).reshape(16, 16)
        _check(lib().hmat_set_tile_table_flags(self._h, int(flagsA), int(flagsB), t.ctypes.data),
               "hmat_set_tile_table_flags")

    def set_fp64_splitk_table(self, table):
        """Install a 16 x 16 FP64 split-k code table (None: built-in rule); see autotune.py."""
        if table is None:
            _check(lib().hmat_set_fp64_splitk_table(self._h, None), "hmat_set_fp64_splitk_table")
            return
        t = np.ascontiguousarray(table, dtype=np.int8).reshape(16, 16)
        _check(lib().hmat_set_fp64_splitk_table(self._h, t.ctypes.data), "hmat_set_fp64_splitk_table")

    def device_error(self) -> int:
        code = _u32()
        _check(lib().hmat_get_device_error(self._h, ctypes.byref(code)), "hmat_get_device_error")
        return code.value


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _mat_args(X, rows, cols, name):
    """(ptr, ld, stride) of an 8 x rows x cols float64 CUDA tensor."""
    import torch
    if X is None:
        return None, max(cols, 1), 0
    if not isinstance(X, torch.Tensor) or X.dtype != torch.float64 or not X.is_cuda:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if X.dim() != 3 or X.shape[0] != 8 or X.shape[1] != rows or X.shape[2] != cols:
        raise ValueError(f"{name} must have shape (8, {rows}, {cols}), got {tuple(X.shape)}")
    if cols > 1 and X.stride(2) != 1:
        raise ValueError(f"{name} components must be row-major (last stride 1)")
    return X.data_ptr(), max(X.stride(1), cols, 1), X.stride(0)


def make_desc(A, B, C, opA="N", opB="N", flagsA=HMAT_BQ, flagsB=HMAT_BQ, alpha=1.0, beta=0.0, m=None, n=None,
              k=None) -> hmat_gemm_desc:
    """A descriptor for C <- alpha op(A) op(B) + beta C over torch tensors."""
    oa, ob = _op(opA), _op(opB)
    ta, tb = oa in (HMAT_OP_T, HMAT_OP_H), ob in (HMAT_OP_T, HMAT_OP_H)
    if m is None:
        m = A.shape[2] if ta else A.shape[1]
    if k is None:
        k = A.shape[1] if ta else A.shape[2]
    if n is None:
        n = B.shape[1] if tb else B.shape[2]
    a_ptr, lda, sa = _mat_args(A, *((k, m) if ta else (m, k)), "A")
    b_ptr, ldb, sb = _mat_args(B, *((n, k) if tb else (k, n)), "B")
    c_ptr, ldc, sc = _mat_args(C, m, n, "C")
    alpha, beta = complex(alpha), complex(beta)
    d = hmat_gemm_desc()
    d.opA, d.opB, d.flagsA, d.flagsB = oa, ob, int(flagsA), int(flagsB)
    d.m, d.n, d.k = int(m), int(n), int(k)
    d.alpha_re, d.alpha_im, d.beta_re, d.beta_im = alpha.real, alpha.imag, beta.real, beta.imag
    d.A, d.lda, d.strideA = a_ptr, lda, sa
    d.B, d.ldb, d.strideB = b_ptr, ldb, sb
    d.C, d.ldc, d.strideC = c_ptr, ldc, sc
    return d


def hmat_workspace_size(handle: Handle, descs, mode="fp64", tol=0.0) -> int:
    arr = (hmat_gemm_desc * len(descs))(*descs)
    out = _sz()
    _check(lib().hmat_workspace_size(handle.value, len(descs), arr, _mode(mode), float(tol), ctypes.byref(out)),
           "hmat_workspace_size")
    return out.value


def _workspace(nbytes, device):
    import torch
    if nbytes == 0:
        return None, 0
    return torch.empty(nbytes, dtype=torch.uint8, device=device), nbytes


def hmat_bq_gemm(handle: Handle, A, B, C, opA="N", opB="N", flagsA=HMAT_BQ, flagsB=HMAT_BQ, alpha=1.0, beta=0.0,
                 mode="fp64", tol=0.0, workspace=None, stream=None):
    """C <- alpha op(A) op(B) + beta C (hmat_bq_gemm); returns C.

    workspace: a uint8 CUDA tensor of at least hmat_workspace_size() bytes, or
    None to allocate one for this call (split mode)."""
    d = make_desc(A, B, C, opA, opB, flagsA, flagsB, alpha, beta)
    md = _mode(mode)
    ws = workspace
    if ws is None:
        ws, _ = _workspace(hmat_workspace_size(handle, [d], md, tol), C.device)
    ws_ptr = ws.data_ptr() if ws is not None else None
    ws_bytes = ws.numel() if ws is not None else 0
    _check(lib().hmat_bq_gemm(handle.value, d.opA, d.opB, d.flagsA, d.flagsB, d.m, d.n, d.k, d.alpha_re,
                              d.alpha_im, d.A, d.lda, d.strideA, d.B, d.ldb, d.strideB, d.beta_re, d.beta_im,
                              d.C, d.ldc, d.strideC, md, float(tol), ws_ptr, ws_bytes, _stream_ptr(stream)),
           "hmat_bq_gemm")
    return C


def hmat_bq_gemm_grouped(handle: Handle, descs, mode="fp64", tol=0.0, workspace=None, stream=None,
                         use_graph=False, device=None):
    """Grouped products (hmat_bq_gemm_grouped) over a list of hmat_gemm_desc."""
    md = _mode(mode)
    arr = (hmat_gemm_desc * len(descs))(*descs)
    ws = workspace
    if ws is None:
        import torch
        ws, _ = _workspace(hmat_workspace_size(handle, descs, md, tol), device or torch.device("cuda"))
    ws_ptr = ws.data_ptr() if ws is not None else None
    ws_bytes = ws.numel() if ws is not None else 0
    st = lib().hmat_bq_gemm_grouped(handle.value, len(descs), arr, md, float(tol), ws_ptr, ws_bytes,
                                    _stream_ptr(stream), 1 if use_graph else 0)
    if st != 0:
        bad = lib().hmat_last_bad_index(handle.value)
        raise HmatError(st, f"hmat_bq_gemm_grouped (descriptor {bad})")


def hmat_workspace_size_modes(handle: Handle, descs, modes, tol=0.0) -> int:
    """Workspace bytes of hmat_bq_gemm_grouped_modes (one mode per descriptor)."""
    if len(modes) != len(descs):
        raise ValueError("one mode per descriptor")
    arr = (hmat_gemm_desc * len(descs))(*descs)
    marr = (_i32 * len(modes))(*[_mode(m) for m in modes])
    out = _sz()
    _check(lib().hmat_workspace_size_modes(handle.value, len(descs), arr, marr, float(tol), ctypes.byref(out)),
           "hmat_workspace_size_modes")
    return out.value


def hmat_bq_gemm_grouped_modes(handle: Handle, descs, modes, tol=0.0, workspace=None, stream=None,
                               use_graph=False, device=None):
    """Grouped products with a mode per product (hmat_bq_gemm_grouped_modes)."""
    if len(modes) != len(descs):
        raise ValueError("one mode per descriptor")
    arr = (hmat_gemm_desc * len(descs))(*descs)
    marr = (_i32 * len(modes))(*[_mode(m) for m in modes])
    ws = workspace
    if ws is None:
        import torch
        ws, _ = _workspace(hmat_workspace_size_modes(handle, descs, modes, tol), device or torch.device("cuda"))
    ws_ptr = ws.data_ptr() if ws is not None else None
    ws_bytes = ws.numel() if ws is not None else 0
    st = lib().hmat_bq_gemm_grouped_modes(handle.value, len(descs), arr, marr, float(tol), ws_ptr, ws_bytes,
                                          _stream_ptr(stream), 1 if use_graph else 0)
    if st != 0:
        bad = lib().hmat_last_bad_index(handle.value)
        raise HmatError(st, f"hmat_bq_gemm_grouped_modes (descriptor {bad})")


def hmat_bq_gemm_split_noalloc(handle: Handle, A, B, C, opA="N", opB="N", flagsA=HMAT_BQ, flagsB=HMAT_BQ,
                               alpha=1.0, beta=0.0, tol=0.0, stream=None):
    """Split-mode product whose workspace is the library's fixed scratch array
    (no allocation by the library or by this binding); returns C.  For callers
    that cannot allocate device memory; limited to small products."""
    d = make_desc(A, B, C, opA, opB, flagsA, flagsB, alpha, beta)
    _check(lib().hmat_bq_gemm_split_noalloc(handle.value, d.opA, d.opB, d.flagsA, d.flagsB, d.m, d.n, d.k,
                                            d.alpha_re, d.alpha_im, d.A, d.lda, d.strideA, d.B, d.ldb, d.strideB,
                                            d.beta_re, d.beta_im, d.C, d.ldc, d.strideC, float(tol),
                                            _stream_ptr(stream)),
           "hmat_bq_gemm_split_noalloc")
    return C


def bq_gemm_host(handle: Handle, A_host, B_host, C_host, opA="N", opB="N", flagsA=HMAT_BQ, flagsB=HMAT_BQ,
                 alpha=1.0, beta=0.0, mode="split", tol=0.0, device_buffers=None, workspace=None, stream=None):
    """End-to-end product on HOST tensors: copy A, B (and C if beta != 0) to the
    device, run hmat_bq_gemm, copy C back.  device_buffers=(dA, dB, dC) reuses
    device storage.  Returns (C_host, h2d_bytes, d2h_bytes)."""
    import torch
    dA, dB, dC = device_buffers if device_buffers is not None else (
        torch.empty_like(A_host, device="cuda"), torch.empty_like(B_host, device="cuda"),
        torch.empty_like(C_host, device="cuda"))
    dA.copy_(A_host, non_blocking=True)
    dB.copy_(B_host, non_blocking=True)
    h2d = A_host.numel() * 8 + B_host.numel() * 8
    if complex(beta) != 0:
        dC.copy_(C_host, non_blocking=True)
        h2d += C_host.numel() * 8
    hmat_bq_gemm(handle, dA, dB, dC, opA, opB, flagsA, flagsB, alpha, beta, mode, tol, workspace, stream)
    C_host.copy_(dC, non_blocking=True)
    return C_host, h2d, C_host.numel() * 8


# ----------------------------------------------------------------------------- streamed (out-of-core) products
def _any_mat_args(X, rows, cols, name):
    """(ptr, ld, stride, on_host) of an 8 x rows x cols float64 tensor on the host or the device."""
    import torch
    if X is None:
        return None, max(cols, 1), 0, False
    if not isinstance(X, torch.Tensor) or X.dtype != torch.float64:
        raise TypeError(f"{name} must be a float64 tensor")
    if X.dim() != 3 or X.shape[0] != 8 or X.shape[1] != rows or X.shape[2] != cols:
        raise ValueError(f"{name} must have shape (8, {rows}, {cols}), got {tuple(X.shape)}")
    if cols > 1 and X.stride(2) != 1:
        raise ValueError(f"{name} components must be row-major (last stride 1)")
    return X.data_ptr(), max(X.stride(1), cols, 1), X.stride(0), not X.is_cuda


def streamed_plan(m, n, k, opA="N", opB="N", flagsA=HMAT_BQ, flagsB=HMAT_BQ, mode="split", tol=0.0,
                  budget=8 << 30, on_host=(True, True, True), handle=None):
    """(mb, nb, kb, device bytes) of the streamed product for a device budget (hmat_streamed_plan)."""
    mb, nb, kb, nbytes = _i64(), _i64(), _i64(), _sz()
    _check(lib().hmat_streamed_plan(handle.value if handle is not None else None, _op(opA), _op(opB), int(flagsA),
                                    int(flagsB), int(m), int(n), int(k), _mode(mode), float(tol), int(budget),
                                    int(on_host[0]), int(on_host[1]), int(on_host[2]), ctypes.byref(mb),
                                    ctypes.byref(nb), ctypes.byref(kb), ctypes.byref(nbytes)), "hmat_streamed_plan")
    return mb.value, nb.value, kb.value, nbytes.value


def streamed_traffic(m, n, k, opA="N", opB="N", flagsA=HMAT_BQ, flagsB=HMAT_BQ, mode="split", tol=0.0,
                     budget=8 << 30, on_host=(True, True, True), beta_nonzero=False, handle=None):
    """(host-to-device, device-to-host) bytes one streamed product copies under that plan
    (hmat_streamed_traffic)."""
    h2d, d2h = _sz(), _sz()
    _check(lib().hmat_streamed_traffic(handle.value if handle is not None else None, _op(opA), _op(opB), int(flagsA),
                                       int(flagsB), int(m), int(n), int(k), _mode(mode), float(tol), int(budget),
                                       int(on_host[0]), int(on_host[1]), int(on_host[2]), int(bool(beta_nonzero)),
                                       ctypes.byref(h2d), ctypes.byref(d2h)), "hmat_streamed_traffic")
    return h2d.value, d2h.value


def hmat_bq_gemm_streamed(handle: Handle, A, B, C, opA="N", opB="N", flagsA=HMAT_BQ, flagsB=HMAT_BQ, alpha=1.0,
                          beta=0.0, mode="split", tol=0.0, budget=None, workspace=None, stream=None):
    """C <- alpha op(A) op(B) + beta C with host (pinned) or device tensors, computed block by block within a
    device budget (hmat_bq_gemm_streamed).  workspace: a uint8 CUDA tensor (the budget), or None to allocate
    `budget` bytes.  Returns C; host buffers are complete once the stream is."""
    import torch
    oa, ob = _op(opA), _op(opB)
    ta, tb = oa in (HMAT_OP_T, HMAT_OP_H), ob in (HMAT_OP_T, HMAT_OP_H)
    m = A.shape[2] if ta else A.shape[1]
    k = A.shape[1] if ta else A.shape[2]
    n = B.shape[1] if tb else B.shape[2]
    a_ptr, lda, sa, _ = _any_mat_args(A, *((k, m) if ta else (m, k)), "A")
    b_ptr, ldb, sb, _ = _any_mat_args(B, *((n, k) if tb else (k, n)), "B")
    c_ptr, ldc, sc, _ = _any_mat_args(C, m, n, "C")
    ws = workspace
    if ws is None:
        if budget is None:
            raise ValueError("give a device budget (bytes) or a workspace tensor")
        ws = torch.empty(int(budget), dtype=torch.uint8, device="cuda")
    alpha, beta = complex(alpha), complex(beta)
    _check(lib().hmat_bq_gemm_streamed(handle.value, oa, ob, int(flagsA), int(flagsB), m, n, k, alpha.real,
                                       alpha.imag, a_ptr, lda, sa, b_ptr, ldb, sb, beta.real, beta.imag, c_ptr, ldc,
                                       sc, _mode(mode), float(tol), ws.data_ptr(), ws.numel(),
                                       _stream_ptr(stream)), "hmat_bq_gemm_streamed")
    return C


# ----------------------------------------------------------------------------- element-wise and mapping operations
def _op_shape(X, op):
    """(rows, cols) of op(X) for a stored 8 x r x c tensor."""
    return (X.shape[2], X.shape[1]) if _op(op) in (HMAT_OP_T, HMAT_OP_H) else (X.shape[1], X.shape[2])


def _cplx_args(Z, rows, cols, name):
    """(ptr, ld in complex elements) of a rows x cols complex128 CUDA tensor (row-major)."""
    import torch
    if not isinstance(Z, torch.Tensor) or Z.dtype != torch.complex128 or not Z.is_cuda:
        raise TypeError(f"{name} must be a complex128 CUDA tensor")
    if Z.dim() != 2 or Z.shape[0] != rows or Z.shape[1] != cols:
        raise ValueError(f"{name} must have shape ({rows}, {cols}), got {tuple(Z.shape)}")
    if cols > 1 and Z.stride(1) != 1:
        raise ValueError(f"{name} must be row-major")
    return Z.data_ptr(), max(Z.stride(0), cols, 1)


def hmat_bq_add(handle: Handle, A, B, C, alpha=1.0, beta=1.0, opA="N", opB="N", flagsA=HMAT_BQ, flagsB=HMAT_BQ,
                stream=None):
    """C <- alpha op(A) + beta op(B) (hmat_bq_add); B may be None.  Returns C."""
    m, n = _op_shape(A, opA)
    ta, tb = _op(opA) in (HMAT_OP_T, HMAT_OP_H), _op(opB) in (HMAT_OP_T, HMAT_OP_H)
    a_ptr, lda, sa = _mat_args(A, *((n, m) if ta else (m, n)), "A")
    b_ptr, ldb, sb = _mat_args(B, *((n, m) if tb else (m, n)), "B")
    c_ptr, ldc, sc = _mat_args(C, m, n, "C")
    alpha, beta = complex(alpha), complex(beta)
    _check(lib().hmat_bq_add(handle.value, _op(opA), _op(opB), int(flagsA), int(flagsB) if B is not None else 0,
                             m, n, alpha.real, alpha.imag, a_ptr, lda, sa, beta.real, beta.imag, b_ptr, ldb, sb,
                             c_ptr, ldc, sc, _stream_ptr(stream)), "hmat_bq_add")
    return C


def hmat_bq_scale(handle: Handle, X, Y, alpha, op="N", flags=HMAT_BQ, stream=None):
    """Y <- alpha op(X) (hmat_bq_scale).  Returns Y."""
    m, n = _op_shape(X, op)
    tr = _op(op) in (HMAT_OP_T, HMAT_OP_H)
    x_ptr, ldx, sx = _mat_args(X, *((n, m) if tr else (m, n)), "X")
    y_ptr, ldy, sy = _mat_args(Y, m, n, "Y")
    alpha = complex(alpha)
    _check(lib().hmat_bq_scale(handle.value, _op(op), int(flags), m, n, alpha.real, alpha.imag, x_ptr, ldx, sx,
                               y_ptr, ldy, sy, _stream_ptr(stream)), "hmat_bq_scale")
    return Y


def hmat_bq_trace(handle: Handle, X, op="N", flags=HMAT_BQ, out=None, stream=None):
    """Tr[op(X)] into a 2-element float64 CUDA tensor (re, im) (hmat_bq_trace); returns it."""
    import torch
    n = X.shape[1]
    x_ptr, ldx, sx = _mat_args(X, n, n, "X")
    if out is None:
        out = torch.empty(2, dtype=torch.float64, device=X.device)
    _check(lib().hmat_bq_trace(handle.value, _op(op), int(flags), n, x_ptr, ldx, sx, out.data_ptr(),
                               _stream_ptr(stream)), "hmat_bq_trace")
    return out


def hmat_bq_to_complex(handle: Handle, X, Z=None, op="N", flags=HMAT_BQ, stream=None):
    """The complex 2m x 2n image of op(X) as a complex128 CUDA tensor (hmat_bq_to_complex)."""
    import torch
    m, n = _op_shape(X, op)
    tr = _op(op) in (HMAT_OP_T, HMAT_OP_H)
    x_ptr, ldx, sx = _mat_args(X, *((n, m) if tr else (m, n)), "X")
    if Z is None:
        Z = torch.empty((2 * m, 2 * n), dtype=torch.complex128, device=X.device)
    z_ptr, ldz = _cplx_args(Z, 2 * m, 2 * n, "Z")
    _check(lib().hmat_bq_to_complex(handle.value, _op(op), int(flags), m, n, x_ptr, ldx, sx, z_ptr, ldz,
                                    _stream_ptr(stream)), "hmat_bq_to_complex")
    return Z


def hmat_complex_to_bq(handle: Handle, Z, Y=None, stream=None):
    """The m x n biquaternion of a 2m x 2n complex128 tensor (hmat_complex_to_bq)."""
    import torch
    m, n = Z.shape[0] // 2, Z.shape[1] // 2
    z_ptr, ldz = _cplx_args(Z, 2 * m, 2 * n, "Z")
    if Y is None:
        Y = torch.empty((8, m, n), dtype=torch.float64, device=Z.device)
    y_ptr, ldy, sy = _mat_args(Y, m, n, "Y")
    _check(lib().hmat_complex_to_bq(handle.value, m, n, z_ptr, ldz, y_ptr, ldy, sy, _stream_ptr(stream)),
           "hmat_complex_to_bq")
    return Y


def hmat_bq_hermiticity(handle: Handle, X, flags=HMAT_BQ, out=None, stream=None):
    """max |X - X^dagger| into a 1-element float64 CUDA tensor (hmat_bq_hermiticity); returns it."""
    import torch
    n = X.shape[1]
    x_ptr, ldx, sx = _mat_args(X, n, n, "X")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=X.device)
    _check(lib().hmat_bq_hermiticity(handle.value, int(flags), n, x_ptr, ldx, sx, out.data_ptr(),
                                     _stream_ptr(stream)), "hmat_bq_hermiticity")
    return out


def hmat_bq_hadamard_block(handle: Handle, X, alpha, flags=0xCC, Z=None, offdiag=True, stream=None):
    """(Z, offdiag) of the Hadamard block reduction (hmat_bq_hadamard_block): Z the n x n complex128
    block, offdiag a 1-element float64 CUDA tensor (or None when offdiag=False)."""
    import torch
    n = X.shape[1]
    x_ptr, ldx, sx = _mat_args(X, n, n, "X")
    if Z is None:
        Z = torch.empty((n, n), dtype=torch.complex128, device=X.device)
    z_ptr, ldz = _cplx_args(Z, n, n, "Z")
    off = torch.empty(1, dtype=torch.float64, device=X.device) if offdiag else None
    a = complex(alpha)
    _check(lib().hmat_bq_hadamard_block(handle.value, int(flags), n, a.real, a.imag, x_ptr, ldx, sx, z_ptr, ldz,
                                        off.data_ptr() if off is not None else None, _stream_ptr(stream)),
           "hmat_bq_hadamard_block")
    return Z, off


__all__ = ["Handle", "HmatError", "hmat_gemm_desc", "hmat_bq_gemm", "hmat_bq_gemm_grouped", "hmat_workspace_size",
           "hmat_bq_gemm_grouped_modes", "hmat_workspace_size_modes",
           "hmat_bq_gemm_split_noalloc", "hmat_bq_gemm_streamed", "streamed_plan", "streamed_traffic", "hmat_bq_add", "hmat_bq_scale", "hmat_bq_trace", "hmat_bq_to_complex",
           "hmat_complex_to_bq", "hmat_bq_hermiticity", "hmat_bq_hadamard_block",
           "bq_gemm_host", "make_desc", "plan_info", "split_info", "lib", "library_path", "OPS", "MODES",
           "CFORMS", "HMAT_REAL", "HMAT_COMPLEX", "HMAT_TRS", "HMAT_TRA", "HMAT_BQ"]
