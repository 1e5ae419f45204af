"""Seeded synthetic input generators (host side, numpy).

This module only produces operand matrices; it holds none of the SpGEMM
arithmetic.  Both the CPU oracle's tests and the CUDA path's tests and bench
draw their inputs from here, so the two sides see identical matrices.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: value(seed, stream, i) = mix(mix(seed + stream*G) + (i+1)*G), with
G the 64-bit golden-ratio increment and mix the SplitMix64 finaliser.

Matrix families follow the paper's test matrices (Section 5.1): R-MAT
(Section 5.1.1, recursive quadrant sampling), Erdos-Renyi (Section 5.1.2, here
with exactly c nonzeros per column at distinct uniform rows) and the 7-point 3D
grid (Section 5.1.3), plus the piecewise-constant aggregation P used for the
multigrid Galerkin product R*A*P (Section 1 and Section 8 name multigrid
restriction and the triple product).
"""
from __future__ import annotations

import os
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

_G = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# semiring tags shared by the whole package (value dtype per semiring)
PLUS_TIMES_F64 = 0
MIN_PLUS_F32 = 1
OR_AND_BOOL = 2
PLUS_TIMES_I64 = 3
SEMIRING_DTYPE = {
    PLUS_TIMES_F64: np.float64,
    MIN_PLUS_F32: np.float32,
    OR_AND_BOOL: np.uint8,
    PLUS_TIMES_I64: np.int64,
}
SEMIRING_NAME = {
    PLUS_TIMES_F64: "plus_times_f64",
    MIN_PLUS_F32: "min_plus_f32",
    OR_AND_BOOL: "or_and_bool",
    PLUS_TIMES_I64: "plus_times_i64",
}


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def u64(seed: int, stream: int, idx) -> np.ndarray:
    """Counter-based SplitMix64 draw for counters ``idx`` of (seed, stream)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        base = _mix(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
                              + np.uint64(stream & 0xFFFFFFFFFFFFFFFF) * _G],
                             dtype=np.uint64))[0]
        return _mix(base + (idx + np.uint64(1)) * _G)


def uniform01(seed: int, stream: int, idx) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits."""
    return (u64(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_int(seed: int, stream: int, idx, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive), by multiply-shift on 32 bits."""
    r = (u64(seed, stream, idx) >> np.uint64(32)).astype(np.uint64)
    span = np.uint64(hi - lo + 1)
    return (lo + ((r * span) >> np.uint64(32)).astype(np.int64)).astype(np.int64)


@dataclass
class CSC:
    """Host CSC matrix: int64 column pointers, int32 row ids sorted per column."""
    m: int
    n: int
    colptr: np.ndarray
    rowidx: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])

    def with_vals(self, vals: np.ndarray) -> "CSC":
        return CSC(self.m, self.n, self.colptr, self.rowidx, vals)


def csc_from_coo(m: int, n: int, rows: np.ndarray, cols: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Pattern of the COO list with duplicates merged, in CSC order."""
    key = cols.astype(np.int64) * np.int64(max(m, 1)) + rows.astype(np.int64)
    key = np.sort(key)   # sorted distinct keys (a plain sort is much faster than np.unique here)
    if len(key) > 1:
        key = key[np.concatenate(([True], key[1:] != key[:-1]))]
    c = key // max(m, 1)
    r = (key - c * max(m, 1)).astype(np.int32)
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(c, minlength=n), out=colptr[1:])
    return colptr, r


def _values(kind: str, seed: int, nnz: int, stream: int = 7777) -> np.ndarray:
    idx = np.arange(nnz, dtype=np.uint64)
    if kind == "f64":
        return uniform01(seed, stream, idx)
    if kind == "f32":
        return uniform01(seed, stream, idx).astype(np.float32)
    if kind == "bool":
        return np.ones(nnz, dtype=np.uint8)
    if kind == "i64":
        return uniform_int(seed, stream, idx, -8, 8)
    raise ValueError(kind)


def values_for(semiring: int, seed: int, nnz: int) -> np.ndarray:
    kind = {PLUS_TIMES_F64: "f64", MIN_PLUS_F32: "f32", OR_AND_BOOL: "bool", PLUS_TIMES_I64: "i64"}[semiring]
    return _values(kind, seed, nnz)


# Large draws are split into chunks of counters that threads fill independently
# (numpy releases the GIL in its array loops).  Every value depends only on its
# counter, so the result does not depend on the chunking or the thread count.
_EDGE_CHUNK = 1 << 20
_pools: dict[str, ThreadPoolExecutor] = {}
_pools_lock = threading.Lock()
_tls = threading.local()


def _pool(name: str) -> ThreadPoolExecutor:
    with _pools_lock:
        p = _pools.get(name)
        if p is None:
            p = ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)))
            _pools[name] = p
        return p


def rmat_edges(scale: int, nedges: int, a: float, b: float, c: float, seed: int,
               first_edge: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """R-MAT edge list: per edge and per level pick a quadrant with probs (a, b, c, d).

    Quadrant a = (row bit 0, col bit 0), b = (0, 1), c = (1, 0), d = (1, 1); bits
    are placed from the most significant end.  No noise, no relabelling.
    """
    rows = np.empty(nedges, dtype=np.int64)
    cols = np.empty(nedges, dtype=np.int64)
    ab, abc = a + b, a + b + c

    def fill(lo: int) -> None:
        hi = min(lo + _EDGE_CHUNK, nedges)
        e = np.arange(first_edge + lo, first_edge + hi, dtype=np.uint64)
        r = np.zeros(hi - lo, dtype=np.int64)
        q = np.zeros(hi - lo, dtype=np.int64)
        for lvl in range(scale):
            u = uniform01(seed, 1 + lvl, e)
            rbit = u >= ab
            cbit = ((u >= a) & (u < ab)) | (u >= abc)
            r = (r << 1) | rbit
            q = (q << 1) | cbit
        rows[lo:hi] = r
        cols[lo:hi] = q

    starts = range(0, nedges, _EDGE_CHUNK)
    if nedges > _EDGE_CHUNK and not getattr(_tls, "serial", False):
        list(_pool("edges").map(fill, starts))
    else:
        for lo in starts:
            fill(lo)
    return rows, cols


def rmat(scale: int, edge_factor: int, seed: int, semiring: int = PLUS_TIMES_F64,
         abc=(0.57, 0.19, 0.19), n: int | None = None) -> CSC:
    """R-MAT matrix with duplicates merged and self-loops kept.

    With ``n`` not a power of two, edges are drawn at scale ceil(log2 n) and
    those with an endpoint >= n are redrawn (drawing continues from the next
    counters) until edge_factor * n edges are kept.  Values are drawn after
    duplicate merging, in CSC order.
    """
    if n is None:
        n = 1 << scale
    want = edge_factor * n
    rows_l, cols_l = [], []
    got, first = 0, 0
    pow2 = n == 1 << scale
    while got < want:
        # the kept edges are the first `want` in counter order, whatever the batch sizes
        batch = want - got if pow2 else max(want - got, 1024) + (want - got) // 2
        r, c = rmat_edges(scale, batch, abc[0], abc[1], abc[2], seed, first)
        first += batch
        keep = (r < n) & (c < n)
        r, c = r[keep], c[keep]
        take = min(len(r), want - got)
        rows_l.append(r[:take])
        cols_l.append(c[:take])
        got += take
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    colptr, rowidx = csc_from_coo(n, n, rows, cols)
    return CSC(n, n, colptr, rowidx, values_for(semiring, seed, len(rowidx)))


def erdos_renyi(m: int, n: int, c: int, seed: int, semiring: int = PLUS_TIMES_F64) -> CSC:
    """Exactly c (<= m) nonzeros per column at distinct uniform rows.

    Each column draws c rows uniformly; a column that drew a repeated row is
    redrawn from the next round's counters (rejection), which gives a uniform
    c-subset.  Rows are sorted, values drawn in CSC order.
    """
    c = min(c, m)
    rows = np.zeros((n, c), dtype=np.int64)
    todo = np.arange(n, dtype=np.int64)
    rnd = 0
    while len(todo) and rnd < 8:
        idx = (todo[:, None] * c + np.arange(c)[None, :]).astype(np.uint64)
        u = uniform01(seed, 100 + rnd, idx)
        r = np.minimum((u * m).astype(np.int64), m - 1)
        r.sort(axis=1)
        rows[todo] = r
        if c > 1:
            bad = np.any(r[:, 1:] == r[:, :-1], axis=1)
        else:
            bad = np.zeros(len(todo), dtype=bool)
        todo = todo[bad]
        rnd += 1
    # columns that keep drawing repeats (c^2 >> m): sequential draws that skip
    # rows already taken, which is sampling without replacement
    for j in todo.tolist():
        taken: list[int] = []
        seen: set[int] = set()
        ctr = 0
        while len(taken) < c:
            u = uniform01(seed, 200, np.arange(ctr, ctr + 2 * c, dtype=np.uint64) + np.uint64(j) * np.uint64(1 << 32))
            ctr += 2 * c
            for r in np.minimum((u * m).astype(np.int64), m - 1).tolist():
                if r not in seen:
                    seen.add(r)
                    taken.append(r)
                    if len(taken) == c:
                        break
        rows[j] = np.sort(np.array(taken, dtype=np.int64))
    colptr = np.arange(0, (n + 1) * c, c, dtype=np.int64)
    rowidx = rows.reshape(-1).astype(np.int32)
    return CSC(m, n, colptr, rowidx, values_for(semiring, seed, len(rowidx)))


def grid3d_laplacian(N: int) -> CSC:
    """7-point Laplacian on an N^3 grid, x fastest: diagonal 6, face neighbours -1."""
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx % N, (idx // N) % N, idx // (N * N)
    rows, cols, vals = [idx], [idx], [np.full(n, 6.0)]
    for d, coord, stride in ((-1, x, 1), (1, x, 1), (-1, y, N), (1, y, N), (-1, z, N * N), (1, z, N * N)):
        ok = (coord + d >= 0) & (coord + d < N)
        rows.append(idx[ok] + d * stride)
        cols.append(idx[ok])
        vals.append(np.full(int(ok.sum()), -1.0))
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((r, c))
    r, c, v = r[order], c[order], v[order]
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(c, minlength=n), out=colptr[1:])
    return CSC(n, n, colptr, r.astype(np.int32), v.astype(np.float64))


def aggregation_2x2x2(N: int) -> CSC:
    """P (N^3 x (N/2)^3): cell (x,y,z) -> aggregate (x/2) + M(y/2) + M^2(z/2), value 1."""
    M = N // 2
    n = N ** 3
    idx = np.arange(n, dtype=np.int64)
    x, y, z = idx % N, (idx // N) % N, idx // (N * N)
    agg = (x // 2) + M * (y // 2) + M * M * (z // 2)
    order = np.lexsort((idx, agg))
    colptr = np.zeros(M ** 3 + 1, dtype=np.int64)
    np.cumsum(np.bincount(agg, minlength=M ** 3), out=colptr[1:])
    return CSC(n, M ** 3, colptr, idx[order].astype(np.int32), np.ones(n, dtype=np.float64))


def restriction(n: int, order: int, seed: int, semiring: int = PLUS_TIMES_F64) -> CSC:
    """Restriction operator S (ceil(n/order) x n, n nonzeros) of a graph contraction of
    the given order (Section 6.2.3): vertex v joins aggregate perm[v] // order for a
    seeded random permutation perm, so every aggregate but the last has `order`
    vertices; S(perm[v] // order, v) = 1."""
    keys = u64(seed, 90, np.arange(n, dtype=np.uint64))
    perm = np.empty(n, dtype=np.int64)
    perm[np.argsort(keys, kind="stable")] = np.arange(n, dtype=np.int64)
    agg = perm // order
    colptr = np.arange(n + 1, dtype=np.int64)   # one nonzero per column v
    one = np.ones(n, dtype=SEMIRING_DTYPE[semiring])
    if semiring == MIN_PLUS_F32:
        one = np.zeros(n, dtype=np.float32)      # the min-plus "one" is 0
    return CSC(-(-n // order), n, colptr, agg.astype(np.int32), one)


def transpose_host(A: CSC) -> CSC:
    """Plain host transpose (used only to build R = P^T as an input)."""
    cols = np.repeat(np.arange(A.n, dtype=np.int64), np.diff(A.colptr))
    rows = A.rowidx.astype(np.int64)
    order = np.lexsort((cols, rows))
    colptr = np.zeros(A.m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=A.m), out=colptr[1:])
    return CSC(A.n, A.m, colptr, cols[order].astype(np.int32), A.vals[order])


def frontier(m: int, k: int, seed: int, lo: int = 1, hi: int = 1000) -> CSC:
    """Tall-skinny BOOL frontier: column j holds round(10^U(log10 lo, log10 hi)) distinct rows."""
    u = uniform01(seed, 50, np.arange(k, dtype=np.uint64))
    cnt = np.clip(np.rint(10.0 ** (np.log10(lo) + u * (np.log10(hi) - np.log10(lo)))), lo, hi).astype(np.int64)
    colptr = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(cnt, out=colptr[1:])
    rows = np.empty(int(colptr[-1]), dtype=np.int32)
    for j in range(k):
        col = erdos_renyi(m, 1, int(cnt[j]), seed * 1315423911 + j, OR_AND_BOOL)
        rows[colptr[j]:colptr[j + 1]] = col.rowidx
    return CSC(m, k, colptr, rows, np.ones(len(rows), dtype=np.uint8))


def batch_pairs(count: int, seed: int, lo_log2: float = 10.0, hi_log2: float = 16.0,
                semiring: int = PLUS_TIMES_I64) -> list[tuple[CSC, CSC]]:
    """Independent uneven pairs (A_i, B_i), n_i = floor(2^U(lo,hi)).

    Each matrix is Erdos-Renyi or R-MAT(0.57, 0.19, 0.19) by coin flip with edge
    factor uniform in {4, 8, 16, 32}; pair i uses seed + i.
    """
    def pair(i: int) -> tuple[CSC, CSC]:
        _tls.serial = True   # pairs are the unit of parallelism here
        s = seed + i
        u = uniform01(s, 60, np.arange(8, dtype=np.uint64))
        n = int(np.floor(2.0 ** (lo_log2 + u[0] * (hi_log2 - lo_log2))))
        mats = []
        for t in range(2):
            ef = (4, 8, 16, 32)[min(int(u[2 + t] * 4), 3)]
            ms = s * 2 + t + 0x51ED
            if u[4 + t] < 0.5:
                mats.append(erdos_renyi(n, n, ef, ms, semiring))
            else:
                scale = max(1, int(np.ceil(np.log2(n))))
                mats.append(rmat(scale, ef, ms, semiring, n=n))
        return mats[0], mats[1]

    return list(_pool("pairs").map(pair, range(count)))


def random_csc(m: int, n: int, density: float, seed: int, semiring: int = PLUS_TIMES_F64) -> CSC:
    """Small Bernoulli(density) pattern for unit tests."""
    idx = np.arange(m * n, dtype=np.uint64)
    keep = uniform01(seed, 70, idx) < density
    flat = np.nonzero(keep)[0]
    cols = flat // max(m, 1)
    rows = flat % max(m, 1)
    colptr, rowidx = csc_from_coo(m, n, rows, cols)
    return CSC(m, n, colptr, rowidx, values_for(semiring, seed, len(rowidx)))


def permutation_matrix(n: int, seed: int, dtype=np.float64) -> tuple[CSC, np.ndarray]:
    """Random permutation matrix Q with Q(perm[j], j) = 1."""
    keys = u64(seed, 80, np.arange(n, dtype=np.uint64))
    perm = np.argsort(keys, kind="stable").astype(np.int64)
    colptr = np.arange(n + 1, dtype=np.int64)
    return CSC(n, n, colptr, perm.astype(np.int32), np.ones(n, dtype=dtype)), perm


def identity(n: int, dtype=np.float64) -> CSC:
    return CSC(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n, dtype=dtype))
