"""Parity of the sort tier (columns of 17 .. 128 products of operands with at most
32,768 rows, sorted in the registers of one warp) with the oracle, at its edges and
just beyond them (129 .. 256 products, the block tier):

* every bin boundary (17, 32, 33, 64, 65, 128, 129, 256 products), each column exactly at it;
* columns whose products come from more than 32 entries of B (most of them hitting
  empty columns of A), so that the products arrive over several chunks of entries;
* heavy duplication (every product of a column on one of three rows) and no
  duplication at all, rows at 0 and at 32767;
* all four semirings, boolean operands with stored false values, int64 cancellation;
* the same columns inside a batch and as SUMMA stage products (bounded slots).
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_matches, check_product, sp
from helpers import DT, MP_F32, OR_BOOL, PT_F64, PT_I64
from paper_1006_2183_gb300.gen import CSC

pytestmark = pytest.mark.gpu
SEMIRINGS = [PT_F64, MP_F32, OR_BOOL, PT_I64]
M = 32768


@pytest.fixture(scope="module")
def ctx():
    return sp().Context()


def _operands(sr, seed):
    """A (M x 600): columns 0..99 empty, 100..399 of 1..8 random rows, 400..499 of 1..3
    rows among {0, 1, 32767}, 500..599 of 1..8 rows in the top 64.  B (600 x n): one
    column per (target flops, style), built greedily from A's column lengths."""
    rng = np.random.default_rng(seed)
    cols = []
    for t in range(600):
        if t < 100:
            rows = np.zeros(0, np.int64)
        elif t < 400:
            rows = rng.choice(M, rng.integers(1, 9), replace=False)
        elif t < 500:
            rows = rng.choice(np.array([0, 1, M - 1]), rng.integers(1, 4), replace=False)
        else:
            rows = M - 64 + rng.choice(64, rng.integers(1, 9), replace=False)
        cols.append(np.sort(rows))
    lens = np.array([len(c) for c in cols])
    colptr = np.zeros(601, np.int64)
    np.cumsum(lens, out=colptr[1:])
    rowidx = np.concatenate(cols).astype(np.int32)
    bcols = []
    for target in (17, 18, 31, 32, 33, 40, 63, 64, 65, 100, 127, 128, 129, 200, 255, 256):
        for style in ("plain", "many_empty", "dups", "top"):
            pool = {"plain": np.arange(100, 400), "many_empty": np.arange(100, 400),
                    "dups": np.arange(400, 500), "top": np.arange(500, 600)}[style]
            ks, f = [], 0
            for k in rng.permutation(pool):
                if f + lens[k] <= target:
                    ks.append(int(k))
                    f += int(lens[k])
                if f == target:
                    break
            if style == "many_empty":
                ks += [int(k) for k in rng.choice(100, 60, replace=False)]
            bcols.append(np.sort(np.array(ks, np.int64)))
    blens = np.array([len(c) for c in bcols])
    bptr = np.zeros(len(bcols) + 1, np.int64)
    np.cumsum(blens, out=bptr[1:])
    bidx = np.concatenate(bcols).astype(np.int32)

    def vals(n, s):
        r = np.random.default_rng(s)
        if sr == PT_F64:
            return r.uniform(-1.0, 1.0, n)
        if sr == MP_F32:
            return r.uniform(0.0, 4.0, n).astype(np.float32)
        if sr == OR_BOOL:
            return (r.random(n) < 0.8).astype(np.uint8)   # stored false values too
        return r.integers(-3, 4, n).astype(np.int64)        # cancellations
    A = CSC(M, 600, colptr, rowidx, vals(len(rowidx), seed + 1).astype(DT[sr]))
    B = CSC(600, len(bcols), bptr, bidx, vals(len(bidx), seed + 2).astype(DT[sr]))
    return A, B


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_sort_tier_edges_flat(ctx, sr):
    A, B = _operands(sr, 0x5A00 + sr)
    fl = oracle.flops_per_col(A, B)
    assert fl.min() >= 17 and fl.max() <= 256 and (fl == 256).any() and (fl == 17).any()
    check_product(ctx, A, B, sr, what="sort tier columns")


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_sort_tier_in_batch_and_summa(ctx, sr):
    s = sp()
    A, B = _operands(sr, 0x5B00 + sr)
    R = oracle.spgemm(A, B, sr)
    dA, dB = s.Matrix.from_host(ctx, A, sr), s.Matrix.from_host(ctx, B, sr)
    Cs = s.spgemm_batch(ctx, [dA, dA], [dB, dB], sr)
    for C in Cs:
        assert_matches(C.to_host(), R, sr, what="batch")
    # a 2 x 2 grid: stage products of row blocks of 16384 rows, into bounded slots
    C = s.spgemm_summa_blocked(ctx, dA, dB, 2, sr)
    assert_matches(C.to_host(), R, sr, what="summa 2 x 2")
