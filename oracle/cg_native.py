"""Oracle, part 3 (Python side): the C/OpenMP CG of ``csr_cg.c`` on the oracle's assembled CSR matrix.

TEST INFRASTRUCTURE ONLY.  Only ``tests/`` and the CPU-baseline legs of ``bench.py`` use it, to time
the oracle's unpreconditioned CG (the solve of K u = b, Sec. 3.1 Eq. lin_system) on several host cores;
``solvers.cg`` is the same recurrence in numpy, and the tests hold the two to the same iterates.

``build()`` compiles ``csr_cg.c`` with gcc and OpenMP into ``oracle/_build/libcsrcg.so`` (plain C, no
architecture flags, so it builds the same way on x86-64 and Arm hosts).
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csr_cg.c")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libcsrcg.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the C CG (gcc -O2 -fopenmp); returns the library path.  Raises RuntimeError on failure."""
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found for the oracle's CG")
    tmp = LIB + ".tmp"
    r = subprocess.run([cc, "-O2", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"], capture_output=True,
                       text=True)
    if r.returncode != 0:
        raise RuntimeError("building the oracle's C CG failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        i64p, i32p, dp = C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_double)
        lib.csr_cg.argtypes = [C.c_int64, i64p, i32p, dp, dp, dp, C.c_double, C.c_int, C.c_int, dp]
        lib.csr_cg.restype = C.c_int
        lib.csr_cg_max_threads.argtypes = []
        lib.csr_cg_max_threads.restype = C.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().csr_cg_max_threads())


class CSR:
    """The oracle's matrix in the index types the C code takes (int64 row pointers, int32 columns)."""

    def __init__(self, K):
        K = sp.csr_matrix(K)
        self.n = K.shape[0]
        self.indptr = np.ascontiguousarray(K.indptr, dtype=np.int64)
        self.indices = np.ascontiguousarray(K.indices, dtype=np.int32)
        self.data = np.ascontiguousarray(K.data, dtype=np.float64)


def cg(K, b, tol=1e-14, maxiter=100000, x0=None, threads=0):
    """Unpreconditioned CG on K u = b (K: scipy matrix or ``CSR``), stopping when ||r||_2 <= tol ||b||_2;
    ``threads`` = OpenMP threads (0 = the default count).  Returns (x, iterations, relative residual)."""
    lib = _load()
    A = K if isinstance(K, CSR) else CSR(K)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    rel = C.c_double()
    dp = C.POINTER(C.c_double)
    it = lib.csr_cg(A.n, A.indptr.ctypes.data_as(C.POINTER(C.c_int64)), A.indices.ctypes.data_as(C.POINTER(C.c_int32)),
                    A.data.ctypes.data_as(dp), b.ctypes.data_as(dp), x.ctypes.data_as(dp), float(tol), int(maxiter),
                    int(threads), C.byref(rel))
    if it < 0:
        raise MemoryError("csr_cg: scratch allocation failed")
    return x, int(it), float(rel.value)
