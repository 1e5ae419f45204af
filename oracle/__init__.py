"""CPU oracle for semiring SpGEMM -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline
and reference legs may import this package.  It shares no code with the CUDA
path (``paper_1006_2183_gb300``) and never imports it.

Contents
  * ``oracle.c`` (loaded through ctypes): Gustavson column-by-column SpGEMM
    with a dense sparse accumulator for the four semirings, the symbolic pass
    and per-column flops.
  * ``formats.py``: CSC -> DCSC (+AUX) conversion, transposition and the 2D
    block split of the virtual Sparse SUMMA grid, written from their
    definitions in numpy.
  * ``features.py`` / ``mlp.py``: the per-column predictor features and a
    float64 forward/backward of the nnz predictor network.
  * ``hgemm.py``: a second, independent formulation of the product, the
    hypersparse outer-product multiply of Section 2.4 (Isect, heap merge).

Parity status of every function is listed in ``PARITY`` below; all are
pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PT_F64, MP_F32, OR_BOOL, PT_I64 = 0, 1, 2, 3
DTYPE = {PT_F64: np.float64, MP_F32: np.float32, OR_BOOL: np.uint8, PT_I64: np.int64}

PARITY = {
    "flops": "pinned: paper's Fig. 8 worked example (19), ER closed form c^2 n, Isect identity",
    "symbolic": "pinned: Fig. 8 pattern (nnz 13), dense brute force, Galerkin closed form",
    "numeric": "pinned: dense brute force (Eq. 1) all semirings, Galerkin closed form values, "
               "transpose/identity/permutation invariants, BFS and 2-hop textbook checks",
    "dcsc": "pinned: the 9x9 example of Figs. 5-7 (JC, CP, IR, NUM, AUX)",
    "partition": "pinned: block reassembly equals the input; block products sum to the flat product",
    "features": "pinned: brute-force per-column sets on small inputs",
    "mlp": "pinned: central finite differences and a closed-form linear case",
    "permute": "pinned: dense definition, inverse permutation, (PAP^T)(PAP^T) = P(AA)P^T",
    "hgemm": "pinned: Fig. 8 Isect, flops identity (19) and pattern; equals the Gustavson oracle",
}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP, no fast-math, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                   "-std=c11", _SRC, "-o", tmp]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.oracle_flops.argtypes = [I64, P, P, P, P]
        lib.oracle_symbolic.argtypes = [I64, P, P, I64, P, P, P, ctypes.c_int]
        lib.oracle_numeric.argtypes = [ctypes.c_int, I64, P, P, P, I64, P, P, P, P, P, P, ctypes.c_int]
        lib.oracle_max_threads.restype = ctypes.c_int
        for f in (lib.oracle_flops, lib.oracle_symbolic, lib.oracle_numeric):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def flops_per_col(A, B) -> np.ndarray:
    """flops_j = sum over k in B(:,j) of nnz(A(:,k))."""
    lib = _load()
    Acp, Bcp, Bir = _c(A.colptr, np.int64), _c(B.colptr, np.int64), _c(B.rowidx, np.int32)
    out = np.zeros(B.n, dtype=np.int64)
    rc = lib.oracle_flops(B.n, _p(Acp), _p(Bcp), _p(Bir), _p(out))
    assert rc == 0
    return out


def symbolic(A, B, nthreads: int = 0) -> np.ndarray:
    """nnz(C(:,j)) for C = A*B (structural)."""
    if A.n != B.m:
        raise ValueError("inner dimensions differ")
    lib = _load()
    Acp, Air = _c(A.colptr, np.int64), _c(A.rowidx, np.int32)
    Bcp, Bir = _c(B.colptr, np.int64), _c(B.rowidx, np.int32)
    out = np.zeros(B.n, dtype=np.int64)
    rc = lib.oracle_symbolic(A.m, _p(Acp), _p(Air), B.n, _p(Bcp), _p(Bir), _p(out), nthreads)
    if rc != 0:
        raise MemoryError("oracle_symbolic failed")
    return out


class OracleCSC:
    """Result container (same attribute names as the generators' CSC)."""

    def __init__(self, m, n, colptr, rowidx, vals):
        self.m, self.n, self.colptr, self.rowidx, self.vals = m, n, colptr, rowidx, vals

    @property
    def nnz(self):
        return int(self.colptr[-1])


def spgemm(A, B, semiring: int, nthreads: int = 0) -> OracleCSC:
    """C = A*B over the semiring; rows sorted ascending within each column."""
    if A.n != B.m:
        raise ValueError("inner dimensions differ")
    lib = _load()
    dt = DTYPE[semiring]
    Acp, Air, Av = _c(A.colptr, np.int64), _c(A.rowidx, np.int32), _c(A.vals, dt)
    Bcp, Bir, Bv = _c(B.colptr, np.int64), _c(B.rowidx, np.int32), _c(B.vals, dt)
    cnt = symbolic(A, B, nthreads)
    Ccp = np.zeros(B.n + 1, dtype=np.int64)
    np.cumsum(cnt, out=Ccp[1:])
    nnz = int(Ccp[-1])
    Cir = np.zeros(max(nnz, 1), dtype=np.int32)
    Cv = np.zeros(max(nnz, 1), dtype=dt)
    rc = lib.oracle_numeric(semiring, A.m, _p(Acp), _p(Air), _p(Av), B.n, _p(Bcp), _p(Bir), _p(Bv),
                            _p(Ccp), _p(Cir), _p(Cv), nthreads)
    if rc != 0:
        raise MemoryError("oracle_numeric failed")
    return OracleCSC(A.m, B.n, Ccp, Cir[:nnz], Cv[:nnz])


def spgemm_columns(A, B, semiring: int, cols: np.ndarray, nthreads: int = 0) -> OracleCSC:
    """Only the listed output columns of A*B (a column-subset of B), for sampled checks."""
    cols = np.asarray(cols, dtype=np.int64)
    lens = B.colptr[cols + 1] - B.colptr[cols]
    cp = np.zeros(len(cols) + 1, dtype=np.int64)
    np.cumsum(lens, out=cp[1:])
    take = np.concatenate([np.arange(B.colptr[c], B.colptr[c + 1]) for c in cols]) if len(cols) else np.zeros(0, np.int64)
    sub = OracleCSC(B.m, len(cols), cp, B.rowidx[take], B.vals[take])
    return spgemm(A, sub, semiring, nthreads)
