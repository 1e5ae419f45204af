"""Second oracle: the hypersparse outer-product multiply of Section 2.4 (Fig. 10).

TEST INFRASTRUCTURE ONLY (same import rule as the rest of ``oracle/``).

The steps, in the paper's order:

1. Transpose B once, so that the rows of B are the columns of B^T.
2. Isect = A.JC intersected with B^T.JC: the indices i for which A(:, i) and
   B(i, :) are both nonempty (the JC arrays are sorted, so a merge of the two
   sorted lists finds them).
3. Each i in Isect stands for a list that is never built: the outer product
   A(:, i) B(i, :), in column-major key order (column of B(i, :) first, then the
   row of A(:, i)).  Its next element is produced on demand.
4. A priority queue (a binary heap) holds the current head of every list; the
   minimum key is taken out repeatedly, added to the last output entry when the
   keys are equal, appended as a new entry otherwise, and replaced by the next
   element of the list it came from.
5. The column-major stack of (row, column, value) is turned into CSC.

Equal keys leave the heap in list order (ascending i) because the list id is the
heap's tie breaker, so every output value is the semiring sum over ascending k,
the order the Gustavson oracle uses; plus-times FP64 is summed plainly here.
Pure Python with heapq: small inputs only.
"""
from __future__ import annotations

import heapq

import numpy as np

from . import formats

PT_F64, MP_F32, OR_BOOL, PT_I64 = 0, 1, 2, 3


def _add(sr, x, y):
    if sr == PT_F64:
        return x + y
    if sr == MP_F32:
        return np.float32(min(x, y))
    if sr == OR_BOOL:
        return 1 if (x or y) else 0
    return (int(x) + int(y) + 2 ** 63) % 2 ** 64 - 2 ** 63


def _mul(sr, a, b):
    if sr == PT_F64:
        return float(a) * float(b)
    if sr == MP_F32:
        return np.float32(np.float32(a) + np.float32(b))
    if sr == OR_BOOL:
        return 1 if (a and b) else 0
    return (int(a) * int(b) + 2 ** 63) % 2 ** 64 - 2 ** 63


def isect(a_colptr, bt_colptr):
    """Sorted indices i with A(:, i) and B^T(:, i) (= B(i, :)) both nonempty."""
    a_jc = formats.to_dcsc(len(a_colptr) - 1, a_colptr)[0]
    b_jc = formats.to_dcsc(len(bt_colptr) - 1, bt_colptr)[0]
    out, p, q = [], 0, 0
    while p < len(a_jc) and q < len(b_jc):
        if a_jc[p] == b_jc[q]:
            out.append(int(a_jc[p]))
            p += 1
            q += 1
        elif a_jc[p] < b_jc[q]:
            p += 1
        else:
            q += 1
    return out


def hgemm(A, B, semiring: int):
    """C = A * B by the heap-merged outer products; returns (colptr, rowidx, vals)."""
    m, k, n = A.m, A.n, B.n
    btcp, btir, btv = formats.transpose(B.m, B.n, B.colptr, B.rowidx, B.vals)   # B^T: n x k
    lists = isect(A.colptr, btcp)
    # list state per i: position in A(:, i) and in B(i, :)
    heap = []
    state = {}
    for li, i in enumerate(lists):
        a0, a1 = int(A.colptr[i]), int(A.colptr[i + 1])
        b0, b1 = int(btcp[i]), int(btcp[i + 1])
        state[li] = [i, a0, a1, a0, b0, b1, b0]
        heapq.heappush(heap, (int(btir[b0]), int(A.rowidx[a0]), li))
    rows, cols, vals = [], [], []
    while heap:
        c, r, li = heapq.heappop(heap)
        i, a0, a1, pa, b0, b1, pb = state[li]
        v = _mul(semiring, A.vals[pa], btv[pb])
        if rows and rows[-1] == r and cols[-1] == c:
            vals[-1] = _add(semiring, vals[-1], v)
        else:
            rows.append(r)
            cols.append(c)
            vals.append(v)
        # next element of list li: the next row of A(:, i), else the next column of B(i, :)
        pa += 1
        if pa == a1:
            pa = a0
            pb += 1
        state[li][3], state[li][6] = pa, pb
        if pb < b1:
            heapq.heappush(heap, (int(btir[pb]), int(A.rowidx[pa]), li))
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(colptr, np.asarray(cols, dtype=np.int64) + 1, 1)
    np.cumsum(colptr, out=colptr)
    dt = np.asarray(A.vals).dtype
    return colptr, np.asarray(rows, dtype=np.int32), np.asarray(vals, dtype=dt)


def flops(A, B) -> int:
    """sum over Isect of nnz(A(:, i)) * nnz(B(i, :)) (the identity of Section 2.4)."""
    btcp = formats.transpose(B.m, B.n, B.colptr, B.rowidx, B.vals)[0]
    return int(sum((A.colptr[i + 1] - A.colptr[i]) * (btcp[i + 1] - btcp[i]) for i in isect(A.colptr, btcp)))
