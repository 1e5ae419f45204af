"""Format oracles (test infrastructure only): DCSC + AUX, transpose, 2D blocks.

DCSC (Section 2.3): a CSC whose column-pointer array is compressed to the
nzc columns that hold a nonzero.  JC lists those column ids in ascending
order, CP (nzc+1 entries) points into IR/NUM, IR and NUM are CSC's row ids and
values unchanged.  AUX (end of Section 2.3) is an index over chunks of
ceil(n/nzc) columns; entry t points to the first nonzero column inside chunk t.
Reading used here (the paper leaves empty chunks open): AUX[t] is the
position in JC of the first nonzero column with id >= t*chunk, so an empty
chunk points at the next chunk's first column, and a final entry holds nzc.
Then the columns of chunk t sit at JC positions [AUX[t], AUX[t+1]).

2D blocks (Section 3.2, Fig. 4; non-divisible dimensions per Section 3.5): a
matrix is split into a g x g grid; block I covers rows [I*mb, min((I+1)*mb, m))
with mb = ceil(m/g) (columns likewise with nb = ceil(n/g)), indices local.
"""
from __future__ import annotations

import numpy as np


def ceil_div(a: int, b: int) -> int:
    return -(-a // b)


def to_dcsc(n: int, colptr: np.ndarray):
    """Return (JC, CP, AUX, chunk) for a CSC with n columns."""
    colptr = np.asarray(colptr, dtype=np.int64)
    lens = colptr[1:] - colptr[:-1]
    jc = np.nonzero(lens > 0)[0].astype(np.int64)
    nzc = len(jc)
    cp = np.concatenate([colptr[jc], colptr[-1:]]).astype(np.int64) if nzc else colptr[-1:].astype(np.int64)
    if n == 0:
        return jc, cp, np.zeros(1, dtype=np.int64), 1
    chunk = ceil_div(n, nzc) if nzc else n
    naux = ceil_div(n, chunk)
    aux = np.empty(naux + 1, dtype=np.int64)
    for t in range(naux):
        # first JC position whose column id >= t*chunk
        aux[t] = int(np.searchsorted(jc, t * chunk, side="left"))
    aux[naux] = nzc
    return jc, cp, aux, chunk


def dcsc_lookup(j: int, jc, cp, aux, chunk):
    """Return the [start, end) range of column j via AUX, or None when empty."""
    t = j // chunk
    for p in range(int(aux[t]), int(aux[t + 1])):
        if jc[p] == j:
            return int(cp[p]), int(cp[p + 1])
    return None


def transpose(m: int, n: int, colptr, rowidx, vals):
    """CSC (m x n) -> CSC of the transpose (n x m), rows sorted."""
    colptr = np.asarray(colptr, dtype=np.int64)
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    rows = np.asarray(rowidx, dtype=np.int64)
    order = np.lexsort((cols, rows))
    tcp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=tcp[1:])
    return tcp, cols[order].astype(np.int32), np.asarray(vals)[order]


def block_ranges(dim: int, g: int):
    b = ceil_div(dim, g) if dim else 0
    return [(min(I * b, dim), min((I + 1) * b, dim)) for I in range(g)]


def extract_block(m: int, n: int, colptr, rowidx, vals, r0: int, r1: int, c0: int, c1: int):
    """CSC of the sub-block rows [r0,r1) x cols [c0,c1) with local indices."""
    colptr = np.asarray(colptr, dtype=np.int64)
    ncols = c1 - c0
    cp = np.zeros(ncols + 1, dtype=np.int64)
    rows_out, vals_out = [], []
    for jj in range(ncols):
        s, e = int(colptr[c0 + jj]), int(colptr[c0 + jj + 1])
        r = np.asarray(rowidx[s:e])
        lo = int(np.searchsorted(r, r0, side="left"))
        hi = int(np.searchsorted(r, r1, side="left"))
        rows_out.append(r[lo:hi] - r0)
        vals_out.append(np.asarray(vals[s + lo:s + hi]))
        cp[jj + 1] = cp[jj] + (hi - lo)
    ir = np.concatenate(rows_out).astype(np.int32) if rows_out else np.zeros(0, np.int32)
    nv = np.concatenate(vals_out) if vals_out else np.zeros(0, np.asarray(vals).dtype)
    return cp, ir, nv


def partition(m: int, n: int, colptr, rowidx, vals, g: int):
    """All g*g blocks as {(I, J): (r0, r1, c0, c1, cp, ir, num)}."""
    out = {}
    rr = block_ranges(m, g)
    cc = block_ranges(n, g)
    for J, (c0, c1) in enumerate(cc):
        for I, (r0, r1) in enumerate(rr):
            cp, ir, nv = extract_block(m, n, colptr, rowidx, vals, r0, r1, c0, c1)
            out[(I, J)] = (r0, r1, c0, c1, cp, ir, nv)
    return out


def permute(m: int, n: int, colptr, rowidx, vals, p, q):
    """B = P A Q^T, i.e. B(p[i], q[j]) = A(i, j): the vertex relabelling of Section
    5.3.3 (C' = (PAP^T)(PBP^T) = PCP^T).  By the definition: every entry moves to
    (p[row], q[col]), then the entries are ordered by (column, row)."""
    cols = np.repeat(np.arange(n, dtype=np.int64), np.diff(colptr))
    r2 = np.asarray(p, dtype=np.int64)[np.asarray(rowidx, dtype=np.int64)]
    c2 = np.asarray(q, dtype=np.int64)[cols]
    order = np.lexsort((r2, c2))
    cp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(c2, minlength=n), out=cp[1:])
    return cp, r2[order].astype(np.int32), np.asarray(vals)[order]
