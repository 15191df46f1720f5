"""CPU oracle for the Strassen path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product library never loads it, and it
shares no code with the CUDA path: it is plain C (``stark_oracle.c``) compiled
with gcc, wrapped here with ctypes and numpy.

Functions (each cites what it follows; see ``stark_oracle.c``):

* ``gemm_classical(A, B)``      -- C = A.B by the definition, k ascending
                                   (Alg. 1's "naive" leaf), float64 or int64
                                   (int64 wraps modulo 2^64).
* ``gemm_rows(A, B, rows)``     -- selected rows of the same product, in float64.
* ``strassen(A, B, depth)``     -- Alg. 1 recursion, C22 with +M3.
* ``strassen_abs(A, B, depth)``  -- the error majorant: Alg. 1 on |A|, |B|
                                   with every sign +, so |dC| <= e * S for
                                   a relative error e per leaf product and
                                   addition.
* ``strassen_operands(X, npad, depth, side)`` -- the divide phase: every leaf's
                                   fp32 operand sum (Alg. 1 / Alg. 3).
* ``split_bf16(x)``, ``split_tf32(x)`` -- hi = RN(x), lo = RN(x - hi) in the
                                   8- / 11-significant-bit formats.
* ``split_fp16(x)``               -- the same in IEEE binary16 (11 bits,
                                   subnormals below 2^-14, overflow to inf).
* ``round_fp16(x)``               -- one binary16 rounding (the pins).
* ``round_sig(x, bits)``        -- one round-to-nearest-even to ``bits``
                                   significant bits.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stark_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source with gcc (plain C, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, vp, ci = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
            lib.oracle_gemm_classical_f64.argtypes = [i64, vp, vp, vp]
            lib.oracle_gemm_classical_i64.argtypes = [i64, vp, vp, vp]
            lib.oracle_gemm_rows_f64.argtypes = [i64, vp, i64, vp, vp, vp]
            lib.oracle_gemm_rows_f32in.argtypes = [i64, vp, i64, vp, vp, vp]
            lib.oracle_strassen_f64.argtypes = [i64, ci, vp, vp, vp]
            lib.oracle_strassen_f64.restype = ci
            lib.oracle_strassen_i64.argtypes = [i64, ci, vp, vp, vp]
            lib.oracle_strassen_i64.restype = ci
            lib.oracle_strassen_abs_f64.argtypes = [i64, ci, vp, vp, vp]
            lib.oracle_strassen_abs_f64.restype = ci
            lib.oracle_strassen_operands_f32.argtypes = [i64, i64, ci, vp, ci, vp]
            lib.oracle_strassen_operands_f32.restype = ci
            lib.oracle_split_bf16.argtypes = [i64, vp, vp, vp]
            lib.oracle_split_tf32.argtypes = [i64, vp, vp, vp]
            lib.oracle_split_fp16.argtypes = [i64, vp, vp, vp]
            lib.oracle_round_fp16_f32.argtypes = [ctypes.c_float]
            lib.oracle_round_fp16_f32.restype = ctypes.c_float
            lib.oracle_round_sig_f32.argtypes = [ctypes.c_float, ci]
            lib.oracle_round_sig_f32.restype = ctypes.c_float
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _square(A: np.ndarray, dtype) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=dtype)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("square 2-D matrix expected")
    return A


def gemm_classical(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """C = A.B by the definition (int64: modulo 2^64; float: float64)."""
    lib = _load()
    if np.issubdtype(np.asarray(A).dtype, np.integer):
        A, B = _square(A, np.int64), _square(B, np.int64)
        C = np.empty_like(A)
        lib.oracle_gemm_classical_i64(A.shape[0], _p(A), _p(B), _p(C))
    else:
        A, B = _square(A, np.float64), _square(B, np.float64)
        C = np.empty_like(A)
        lib.oracle_gemm_classical_f64(A.shape[0], _p(A), _p(B), _p(C))
    return C


def gemm_rows(A: np.ndarray, B: np.ndarray, rows) -> np.ndarray:
    """Rows ``rows`` of A.B in float64 (fp32 inputs are widened exactly)."""
    lib = _load()
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    if np.asarray(A).dtype == np.float32:
        A, B = _square(A, np.float32), _square(B, np.float32)
        fn = lib.oracle_gemm_rows_f32in
    else:
        A, B = _square(A, np.float64), _square(B, np.float64)
        fn = lib.oracle_gemm_rows_f64
    n = A.shape[0]
    if rows.size and (rows.min() < 0 or rows.max() >= n):
        raise ValueError("row index out of range")
    out = np.empty((rows.size, n), dtype=np.float64)
    fn(n, _p(rows), rows.size, _p(A), _p(B), _p(out))
    return out


def strassen(A: np.ndarray, B: np.ndarray, depth: int) -> np.ndarray:
    """Alg. 1 with ``depth`` recursion levels (C22 = M1 - M2 + M3 + M6)."""
    lib = _load()
    if np.issubdtype(np.asarray(A).dtype, np.integer):
        A, B = _square(A, np.int64), _square(B, np.int64)
        C = np.empty_like(A)
        rc = lib.oracle_strassen_i64(A.shape[0], depth, _p(A), _p(B), _p(C))
    else:
        A, B = _square(A, np.float64), _square(B, np.float64)
        C = np.empty_like(A)
        rc = lib.oracle_strassen_f64(A.shape[0], depth, _p(A), _p(B), _p(C))
    if rc != 0:
        raise ValueError("oracle strassen rejected its arguments")
    return C


def strassen_abs(A: np.ndarray, B: np.ndarray, depth: int) -> np.ndarray:
    """Error majorant S of Alg. 1 with ``depth`` levels: the recursion on
    |A| and |B| with every coefficient +1 (float64)."""
    lib = _load()
    A, B = _square(A, np.float64), _square(B, np.float64)
    S = np.empty_like(A)
    if lib.oracle_strassen_abs_f64(A.shape[0], depth, _p(A), _p(B), _p(S)) != 0:
        raise ValueError("oracle strassen_abs rejected its arguments")
    return S


def strassen_operands(X: np.ndarray, npad: int, depth: int, side: str) -> np.ndarray:
    """fp32 leaf operand sums, shape (7**depth, npad/2**depth, npad/2**depth).

    ``side`` is ``"A"`` (the A_ij sums of M1..M7) or ``"B"``.  X is read as the
    zero-padded ``npad x npad`` matrix."""
    lib = _load()
    X = _square(X, np.float32)
    L = npad >> depth
    out = np.empty((7 ** depth, L, L), dtype=np.float32)
    rc = lib.oracle_strassen_operands_f32(X.shape[0], npad, depth, _p(X), 0 if side == "A" else 1, _p(out))
    if rc != 0:
        raise ValueError("oracle divide rejected its arguments")
    return out


def split_bf16(x: np.ndarray):
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    hi, lo = np.empty_like(x), np.empty_like(x)
    lib.oracle_split_bf16(x.size, _p(x), _p(hi), _p(lo))
    return hi, lo


def split_tf32(x: np.ndarray):
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    hi, lo = np.empty_like(x), np.empty_like(x)
    lib.oracle_split_tf32(x.size, _p(x), _p(hi), _p(lo))
    return hi, lo


def split_fp16(x: np.ndarray):
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    hi, lo = np.empty_like(x), np.empty_like(x)
    lib.oracle_split_fp16(x.size, _p(x), _p(hi), _p(lo))
    return hi, lo


def round_fp16(x: float) -> float:
    return float(_load().oracle_round_fp16_f32(ctypes.c_float(x)))


def round_sig(x: float, bits: int) -> float:
    return float(_load().oracle_round_sig_f32(ctypes.c_float(x), bits))
