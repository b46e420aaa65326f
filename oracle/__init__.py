"""CPU oracle for C = A*B -- TEST INFRASTRUCTURE, not part of the library.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package. It shares no code with the GPU library:

* ``mm_oracle.c``  the paper's FP64 triple loop (Sec. III definition, Sec. V
  serial program, Sec. III-A-1 OpenMP scheme) and |A||B| for the error bound;
* ``emulation.py`` the split-precision modes written from the published
  splitting methods (numpy, integer-exact);
* ``cpu_variants.c`` the paper's column-prefetching and cache-tiling forms of
  the loop (Sec. III), for extra CPU-baseline rows; same values as the oracle.

``build()`` compiles ``mm_oracle.c`` into ``oracle/_build/libmm_oracle.so`` with
gcc (-O2 -ffp-contract=off, OpenMP). Parity status: every function here is
pinned by ``tests/test_oracle_*.py`` (closed forms, exactness, brute force);
none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmm_oracle.so")
_SRC = os.path.join(_HERE, "mm_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "cpu_variants.c")]
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc; portable C, no intrinsics)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or any(os.path.getmtime(_SO) < os.path.getmtime(f) for f in _SRCS):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp] + _SRCS
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        i64, P = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        for name in ("oracle_gemm", "oracle_absprod"):
            getattr(lib, name).argtypes = [i64, i64, i64, P, i64, P, i64, P, i64]
            getattr(lib, name).restype = None
        for name in ("oracle_gemm_rows", "oracle_absprod_rows"):
            getattr(lib, name).argtypes = [i64, i64, i64, i64, P, i64, P, i64, P, i64]
            getattr(lib, name).restype = None
        for name in ("oracle_gemm_omp", "oracle_absprod_omp", "cpu_gemm_colprefetch", "cpu_gemm_tiled"):
            getattr(lib, name).argtypes = [i64, i64, i64, i64, P, i64, P, i64, P, i64, ctypes.c_int]
            getattr(lib, name).restype = ctypes.c_int
        lib.oracle_dot.argtypes = [i64, i64, i64, P, i64, P, i64]
        lib.oracle_dot.restype = ctypes.c_double
        _lib = lib
    return _lib


def _p(x):
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _prep(A, B):
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    if A.ndim != 2 or B.ndim != 2 or A.shape[1] != B.shape[0]:
        raise ValueError("shapes do not chain")
    return A, B


def gemm(A, B) -> np.ndarray:
    """C = A*B by the serial i-j-k triple loop, k ascending, no FMA."""
    A, B = _prep(A, B)
    m, k = A.shape
    n = B.shape[1]
    C = np.zeros((m, n))
    if m and n:
        _load().oracle_gemm(m, n, k, _p(A), max(k, 1), _p(B), max(n, 1), _p(C), max(n, 1))
    return C


def gemm_rows(A, B, rows) -> np.ndarray:
    """Rows `rows` (a sequence of indices) of A*B, each by the triple loop."""
    A, B = _prep(A, B)
    k, n = B.shape
    out = np.zeros((len(rows), n))
    lib = _load()
    for r, i in enumerate(rows):
        row = out[r]
        lib.oracle_gemm_rows(int(i), int(i) + 1, n, k, _p(A), max(k, 1), _p(B), max(n, 1),
                             _p(row), max(n, 1))
    return out


def absprod(A, B) -> np.ndarray:
    """|A|*|B| by the same loop (scale of the componentwise bound)."""
    A, B = _prep(A, B)
    m, k = A.shape
    n = B.shape[1]
    D = np.zeros((m, n))
    if m and n:
        _load().oracle_absprod(m, n, k, _p(A), max(k, 1), _p(B), max(n, 1), _p(D), max(n, 1))
    return D


def absprod_rows(A, B, rows) -> np.ndarray:
    """Rows `rows` of |A|*|B|."""
    A, B = _prep(A, B)
    k, n = B.shape
    out = np.zeros((len(rows), n))
    lib = _load()
    for r, i in enumerate(rows):
        row = out[r]
        lib.oracle_absprod_rows(int(i), int(i) + 1, n, k, _p(A), max(k, 1), _p(B), max(n, 1),
                                _p(row), max(n, 1))
    return out


def dot(A, B, i: int, j: int) -> float:
    """One element C[i][j]."""
    A, B = _prep(A, B)
    return _load().oracle_dot(i, j, A.shape[1], _p(A), max(A.shape[1], 1), _p(B), max(B.shape[1], 1))


def gemm_omp_rows(A, B, r0: int, r1: int, nthreads: int = 0):
    """Rows [r0, r1) by the OpenMP parallel-for variant; returns (C_rows, threads)."""
    A, B = _prep(A, B)
    k, n = B.shape
    out = np.zeros((r1 - r0, n))
    used = _load().oracle_gemm_omp(r0, r1, n, k, _p(A), max(k, 1), _p(B), max(n, 1),
                                   _p(out), max(n, 1), nthreads)
    return out, used


def gemm_rows_par(A, B, rows) -> np.ndarray:
    """Rows `rows` of A*B by the OpenMP row loop (each element the serial
    triple loop's, bit for bit), for sampled rows of large products."""
    A, B = _prep(A, B)
    As = np.ascontiguousarray(A[list(rows)])
    out, _ = gemm_omp_rows(As, B, 0, As.shape[0])
    return out


def absprod_rows_par(A, B, rows) -> np.ndarray:
    """Rows `rows` of |A|*|B| by the OpenMP row loop."""
    A, B = _prep(A, B)
    As = np.ascontiguousarray(A[list(rows)])
    k, n = B.shape
    out = np.zeros((As.shape[0], n))
    if As.shape[0] and n:
        _load().oracle_absprod_omp(0, As.shape[0], n, k, _p(As), max(k, 1), _p(B), max(n, 1), _p(out), max(n, 1), 0)
    return out


def _rows_variant(fn, A, B, r0, r1, nthreads):
    A, B = _prep(A, B)
    k, n = B.shape
    out = np.zeros((r1 - r0, n))
    used = fn(r0, r1, n, k, _p(A), max(k, 1), _p(B), max(n, 1), _p(out), max(n, 1), nthreads)
    if used <= 0:
        raise MemoryError("cpu variant could not allocate its buffer")
    return out, used


def gemm_colprefetch_rows(A, B, r0: int, r1: int, nthreads: int = 0):
    """Rows [r0, r1) with column prefetching (Sec. III), OpenMP; (C_rows, threads)."""
    return _rows_variant(_load().cpu_gemm_colprefetch, A, B, r0, r1, nthreads)


def gemm_tiled_rows(A, B, r0: int, r1: int, nthreads: int = 0):
    """Rows [r0, r1) with cache tiling (Sec. III), OpenMP; (C_rows, threads)."""
    return _rows_variant(_load().cpu_gemm_tiled, A, B, r0, r1, nthreads)

