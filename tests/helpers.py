"""Test helpers: dense brute force (Eq. 1), golden-file parsing, CSC comparisons."""
from __future__ import annotations

import os

import numpy as np

from paper_1006_2183_gb300.gen import CSC

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

PT_F64, MP_F32, OR_BOOL, PT_I64 = 0, 1, 2, 3
DT = {PT_F64: np.float64, MP_F32: np.float32, OR_BOOL: np.uint8, PT_I64: np.int64}
FP64_RTOL = 1e-13


def dense_bruteforce(A: CSC, B: CSC, sr: int):
    """Inner-product definition (Eq. 1) on dense arrays with structure masks.

    C(i,j) = (+)_l A(i,l) (x) B(l,j) over the l where both entries are stored;
    the entry exists iff at least one such l exists.  Pure Python loops, tiny
    sizes only.
    """
    m, k, n = A.m, A.n, B.n
    Ad = {}
    for j in range(A.n):
        for p in range(A.colptr[j], A.colptr[j + 1]):
            Ad[(int(A.rowidx[p]), j)] = A.vals[p]
    Bd = {}
    for j in range(B.n):
        for p in range(B.colptr[j], B.colptr[j + 1]):
            Bd[(int(B.rowidx[p]), j)] = B.vals[p]
    out = {}
    for i in range(m):
        for j in range(n):
            acc = None
            for l in range(k):
                if (i, l) in Ad and (l, j) in Bd:
                    a, b = Ad[(i, l)], Bd[(l, j)]
                    if sr == PT_F64:
                        x = float(a) * float(b)
                        acc = x if acc is None else acc + x
                    elif sr == MP_F32:
                        x = np.float32(np.float32(a) + np.float32(b))
                        acc = x if acc is None else min(acc, x)
                    elif sr == OR_BOOL:
                        x = int(bool(a) and bool(b))
                        acc = x if acc is None else (acc | x)
                    else:
                        x = (int(a) * int(b))
                        acc = x if acc is None else acc + x
            if acc is not None:
                out[(i, j)] = acc
    return out


def csc_to_dict(C) -> dict:
    d = {}
    for j in range(C.n):
        for p in range(int(C.colptr[j]), int(C.colptr[j + 1])):
            d[(int(C.rowidx[p]), j)] = C.vals[p]
    return d


def assert_sorted_unique(C):
    for j in range(C.n):
        r = np.asarray(C.rowidx[C.colptr[j]:C.colptr[j + 1]])
        assert np.all(r[1:] > r[:-1]), f"column {j} rows not strictly ascending"


def assert_csc_equal(X, Y, sr: int, rtol: float = FP64_RTOL):
    """Structure bit-exact; values bit-exact except plus-times FP64 (relative rtol)."""
    assert X.m == Y.m and X.n == Y.n
    np.testing.assert_array_equal(np.asarray(X.colptr, np.int64), np.asarray(Y.colptr, np.int64))
    np.testing.assert_array_equal(np.asarray(X.rowidx, np.int32), np.asarray(Y.rowidx, np.int32))
    xv, yv = np.asarray(X.vals), np.asarray(Y.vals)
    if sr == PT_F64:
        err = np.abs(xv - yv)
        bound = rtol * np.abs(yv)
        bad = err > bound
        assert not bad.any(), f"{bad.sum()} entries beyond rtol {rtol}: max rel {np.max(err / np.maximum(np.abs(yv), 1e-300))}"
    else:
        np.testing.assert_array_equal(xv, yv)


def read_golden(name: str) -> list[str]:
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.rstrip("\n") for ln in f if ln.strip() and not ln.startswith("#")]


def pattern_matrix(rows_of: dict, m: int, n: int, by_row: bool, sr: int = PT_F64, seed: int = 0) -> CSC:
    """CSC from a {line index: [indices]} pattern (1-based), values 1 + small seeded integers."""
    cols_l, rows_l = [], []
    for a, lst in rows_of.items():
        for b in lst:
            if by_row:
                rows_l.append(a - 1); cols_l.append(b - 1)
            else:
                cols_l.append(a - 1); rows_l.append(b - 1)
    key = np.array(cols_l, np.int64) * m + np.array(rows_l, np.int64)
    key = np.sort(key)
    c = key // m
    r = (key % m).astype(np.int32)
    colptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(c, minlength=n), out=colptr[1:])
    vals = (1 + (np.arange(len(r)) * 7 + seed) % 5).astype(DT[sr])
    return CSC(m, n, colptr, r, vals)
