"""Per-column predictor features, written from their definitions (test infrastructure only).

The paper has no predictor; its Section 8 names structure prediction as
future work.  The features below are this library's own definition of what the
nnz(C(:,j)) predictor sees for an output column j of C = A*B:

  d_j      = nnz(B(:,j))
  flops_j  = sum_{k in B(:,j)} len_k,   len_k = nnz(A(:,k))
  max_j    = max_{k in B(:,j)} len_k     (a lower bound on nnz(C(:,j)))
  sketch_j = OR_{k in B(:,j)} sketch(A(:,k)),  sketch(A(:,k)) = OR_i 2^h(i),
             h(i) = bits 31..26 of the 32-bit product i * 0x9E3779B1
  pc_j     = popcount(sketch_j);  lc_j = 64 ln(64 / (64 - min(pc_j, 63.5)))
             (linear counting, Whang, Vander-Zanden & Taylor 1990)

and the network input x_j (8 floats) is
  [log1p d, log1p flops, log1p max, log1p m, log1p lc, log1p min(flops, m),
   log1p(flops - max), pc / 64].
"""
from __future__ import annotations

import math

import numpy as np


def row_hash_bit(i: np.ndarray) -> np.ndarray:
    h = (np.asarray(i, dtype=np.uint64) * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)
    return (h >> np.uint64(26)).astype(np.uint64)


def column_sketches(A) -> np.ndarray:
    """sketch(A(:,k)) for every column k, by brute force over each column's rows."""
    sk = np.zeros(A.n, dtype=np.uint64)
    bits = np.uint64(1) << row_hash_bit(A.rowidx)
    for k in range(A.n):
        s, e = int(A.colptr[k]), int(A.colptr[k + 1])
        v = np.uint64(0)
        for b in bits[s:e]:
            v |= b
        sk[k] = v
    return sk


def raw_features(A, B, cols=None):
    """(d, flops, maxlen, pc) per listed output column, by direct loops."""
    lens = np.diff(np.asarray(A.colptr, dtype=np.int64))
    sk = column_sketches(A)
    cols = range(B.n) if cols is None else cols
    d, fl, mx, pc = [], [], [], []
    for j in cols:
        s, e = int(B.colptr[j]), int(B.colptr[j + 1])
        ks = np.asarray(B.rowidx[s:e], dtype=np.int64)
        d.append(e - s)
        fl.append(int(lens[ks].sum()) if len(ks) else 0)
        mx.append(int(lens[ks].max()) if len(ks) else 0)
        v = 0
        for k in ks:
            v |= int(sk[k])
        pc.append(bin(v).count("1"))
    return (np.array(d, np.int64), np.array(fl, np.int64), np.array(mx, np.int64), np.array(pc, np.int64))


def feature_vector(d, flops, maxlen, pc, m) -> np.ndarray:
    """The 8 network inputs per column (float64), from the raw counts."""
    d = np.asarray(d, np.float64)
    flops = np.asarray(flops, np.float64)
    maxlen = np.asarray(maxlen, np.float64)
    pcf = np.minimum(np.asarray(pc, np.float64), 63.5)
    lc = 64.0 * np.log(64.0 / (64.0 - pcf))
    x = np.stack([
        np.log1p(d),
        np.log1p(flops),
        np.log1p(maxlen),
        np.full_like(d, math.log1p(m)),
        np.log1p(lc),
        np.log1p(np.minimum(flops, float(m))),
        np.log1p(flops - maxlen),
        np.asarray(pc, np.float64) / 64.0,
    ], axis=1)
    return x
