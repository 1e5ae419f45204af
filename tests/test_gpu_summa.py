"""Parity of the virtual 2D Sparse SUMMA (g x g DCSC blocks, stage products, stage merge) with the oracle.

Blocking changes only the order of the (+) reductions, so structure and the
three exact semirings must match the oracle bit for bit, plus-times FP64
within 1e-13 relative (Sections 3.2, 3.5, 5.3).
"""
import numpy as np
import pytest

import oracle
from oracle import formats as of
from gpu_util import assert_matches, sp
from helpers import MP_F32, OR_BOOL, PT_F64, PT_I64
from paper_1006_2183_gb300 import gen
from paper_1006_2183_gb300.gen import CSC

pytestmark = pytest.mark.gpu
SEMIRINGS = [PT_F64, MP_F32, OR_BOOL, PT_I64]


@pytest.fixture(scope="module")
def ctx():
    return sp().Context()


def blocked(ctx, A, B, sr, g, **kw):
    s = sp()
    dA = s.Matrix.from_host(ctx, A, sr)
    dB = dA if B is A else s.Matrix.from_host(ctx, B, sr)
    return s.spgemm_summa_blocked(ctx, dA, dB, g, sr, s.default_opts(**kw) if kw else None).to_host()


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_summa_rectangular_ragged(ctx, sr):
    for t, (m, k, n, d, g) in enumerate([(37, 29, 41, 0.1, 4), (100, 64, 90, 0.05, 7), (5, 3, 2, 0.6, 4),
                                         (300, 200, 150, 0.03, 16), (1, 20, 30, 0.3, 3)]):
        A = gen.random_csc(m, k, d, 300 + t, sr)
        B = gen.random_csc(k, n, d, 400 + t, sr)
        R = oracle.spgemm(A, B, sr)
        C = blocked(ctx, A, B, sr, g)
        assert_matches(C, R, sr, what=f"{(m, k, n, g)}")


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_summa_rmat_grid16(ctx, sr):
    A = gen.rmat(12, 8, 0x1216, sr)
    R = oracle.spgemm(A, A, sr)
    assert_matches(blocked(ctx, A, A, sr, 16), R, sr)


@pytest.mark.parametrize("every", [1, 3])
def test_summa_merge_every_same_result(ctx, every):
    sr = PT_I64
    A = gen.rmat(11, 8, 0x1108, sr)
    R = oracle.spgemm(A, A, sr)
    assert_matches(blocked(ctx, A, A, sr, 8, summa_merge_every=every), R, sr, what=f"every {every}")


def test_summa_g1_equals_flat(ctx):
    A = gen.erdos_renyi(4096, 4096, 8, 0x1001)
    R = oracle.spgemm(A, A, PT_F64)
    assert_matches(blocked(ctx, A, A, PT_F64, 1), R, PT_F64)


def test_summa_stats_match_block_flops(ctx):
    s = sp()
    sr = PT_I64
    g = 6
    A = gen.random_csc(70, 50, 0.08, 91, sr)
    B = gen.random_csc(50, 60, 0.08, 92, sr)
    blocked(ctx, A, B, sr, g)
    stage_flops, nonempty = s.spgemm_summa_stats(ctx, g)
    bA = of.partition(A.m, A.n, A.colptr, A.rowidx, A.vals, g)
    bB = of.partition(B.m, B.n, B.colptr, B.rowidx, B.vals, g)
    want = [0] * g
    cnt = 0
    for st in range(g):
        for I in range(g):
            for J in range(g):
                r0, r1, k0, k1, cpa, ira, nva = bA[(I, st)]
                _, _, c0, c1, cpb, irb, nvb = bB[(st, J)]
                if len(ira) == 0 or len(irb) == 0:
                    continue
                cnt += 1
                Ab = CSC(r1 - r0, k1 - k0, cpa, ira, nva)
                Bb = CSC(k1 - k0, c1 - c0, cpb, irb, nvb)
                want[st] += int(oracle.flops_per_col(Ab, Bb).sum())
    assert stage_flops == want
    assert nonempty == cnt
    assert sum(stage_flops) == int(oracle.flops_per_col(A, B).sum())


def test_summa_empty_and_errors(ctx):
    s = sp()
    Z = CSC(9, 7, np.zeros(8, np.int64), np.zeros(0, np.int32), np.zeros(0))
    Y = CSC(7, 5, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0))
    C = blocked(ctx, Z, Y, PT_F64, 4)
    assert C.nnz == 0 and list(C.colptr) == [0] * 6
    A = gen.random_csc(10, 8, 0.3, 1)
    dA = s.Matrix.from_host(ctx, A, PT_F64)
    with pytest.raises(s.SpGEMMError):
        s.spgemm_summa_blocked(ctx, dA, dA, 4, PT_F64)   # 10 x 8 times 10 x 8
    B = gen.random_csc(8, 8, 0.3, 2)
    dB = s.Matrix.from_host(ctx, B, PT_F64)
    with pytest.raises(s.SpGEMMError):
        s.spgemm_summa_blocked(ctx, dA, dB, 0, PT_F64)
    # a row index past m: the block split reports it instead of writing past its blocks
    bad = B.rowidx.copy()
    bad[len(bad) // 2] = B.m + 5
    dbad = s.Matrix.from_host(ctx, CSC(B.m, B.n, B.colptr, bad, B.vals), PT_F64)
    with pytest.raises(s.SpGEMMError) as ei:
        s.spgemm_summa_blocked(ctx, dbad, dB, 4, PT_F64)
    assert ei.value.status == 3   # SPGEMM_ERR_BAD_FORMAT
    C = blocked(ctx, B, B, PT_F64, 4)   # the context still works
    assert_matches(C, oracle.spgemm(B, B, PT_F64), PT_F64, what="after bad format")


@pytest.mark.parametrize("sr", [PT_F64, MP_F32])
def test_summa_scale18_sampled(ctx, sr):
    """The secondary benchmark workload: R-MAT scale 18 on a 16 x 16 grid in plus-times
    FP64 and min-plus FP32 (the bench's two semirings there); all column counts vs the
    oracle's symbolic pass and sampled columns vs the oracle (min-plus bit-exact)."""
    A = gen.rmat(18, 8, 0x1802, PT_F64)
    if sr == MP_F32:
        A = A.with_vals(A.vals.astype(np.float32))   # the bench's FP32 rounding of the same values
    C = blocked(ctx, A, A, sr, 16)
    np.testing.assert_array_equal(np.diff(C.colptr), oracle.symbolic(A, A))
    rng = np.random.default_rng(3)
    lens = np.diff(A.colptr)
    cols = np.unique(np.concatenate([np.argsort(lens)[-10:], rng.choice(A.n, 200, replace=False)]))
    R = oracle.spgemm_columns(A, A, sr, cols)
    for t, j in enumerate(cols):
        np.testing.assert_array_equal(C.rowidx[C.colptr[j]:C.colptr[j + 1]], R.rowidx[R.colptr[t]:R.colptr[t + 1]])
        got = C.vals[C.colptr[j]:C.colptr[j + 1]]
        ref = R.vals[R.colptr[t]:R.colptr[t + 1]]
        if sr == PT_F64:
            assert np.all(np.abs(got - ref) <= 1e-13 * np.abs(ref)), j
        else:
            np.testing.assert_array_equal(got, ref, err_msg=f"column {j}")


@pytest.mark.parametrize("g", [4, 7, 16])
def test_summa_block_flops_match_oracle(ctx, g):
    """Per-block work flops(A(I,s) * B(s,J)) against the oracle's block split, and
    their sum against the flat flops (Section 7.1's load-imbalance input)."""
    s = sp()
    A = gen.rmat(11, 8, 0x7101, PT_F64)
    B = gen.erdos_renyi(A.n, 300, 5, 0x7102, PT_F64)
    got = s.spgemm_summa_block_flops(ctx, s.Matrix.from_host(ctx, A, PT_F64), s.Matrix.from_host(ctx, B, PT_F64), g)
    ba = of.partition(A.m, A.n, A.colptr, A.rowidx, A.vals, g)
    bb = of.partition(B.m, B.n, B.colptr, B.rowidx, B.vals, g)
    want = np.zeros((g, g, g), np.int64)
    for st in range(g):
        for J in range(g):
            for I in range(g):
                r0, r1, c0, c1, cpa, ira, va = ba[(I, st)]
                s0, s1, d0, d1, cpb, irb, vb = bb[(st, J)]
                Ab = CSC(r1 - r0, c1 - c0, cpa, ira, va)
                Bb = CSC(s1 - s0, d1 - d0, cpb, irb, vb)
                if Ab.n and Bb.n:
                    want[st, J, I] = int(oracle.flops_per_col(Ab, Bb).sum())
    np.testing.assert_array_equal(got, want)
    assert got.sum() == int(oracle.flops_per_col(A, B).sum())


@pytest.mark.parametrize("sr", [PT_I64, OR_BOOL])
def test_random_symmetric_permutation(ctx, sr):
    """A' = P A P^T on the device equals the oracle's permutation, and
    A'A' = P (AA) P^T exactly, flat and on the grid (Section 5.3.3)."""
    import torch
    s = sp()
    A = gen.rmat(13, 8, 0x7201, sr)
    p = np.random.default_rng(0x7202).permutation(A.n).astype(np.int32)
    pd = torch.from_numpy(p).to(ctx.device)
    dA = s.Matrix.from_host(ctx, A, sr)
    dAp = s.spgemm_mat_permute(ctx, dA, pd, pd)
    ref = of.permute(A.m, A.n, A.colptr, A.rowidx, A.vals, p, p)
    Ap = dAp.to_host()
    np.testing.assert_array_equal(Ap.colptr, ref[0])
    np.testing.assert_array_equal(Ap.rowidx, ref[1])
    np.testing.assert_array_equal(Ap.vals, ref[2])
    C = s.spgemm_multiply(ctx, dA, dA, sr)
    Cperm = s.spgemm_mat_permute(ctx, C, pd, pd).to_host()
    for Cp in (s.spgemm_multiply(ctx, dAp, dAp, sr).to_host(), s.spgemm_summa_blocked(ctx, dAp, dAp, 16, sr).to_host()):
        assert_matches(Cp, Cperm, sr)
    # a rectangular permutation with different row and column maps
    B = gen.random_csc(300, 170, 0.05, 0x7203, sr)
    pr = np.random.default_rng(1).permutation(300).astype(np.int32)
    pc = np.random.default_rng(2).permutation(170).astype(np.int32)
    got = s.spgemm_mat_permute(ctx, s.Matrix.from_host(ctx, B, sr), torch.from_numpy(pr).to(ctx.device),
                               torch.from_numpy(pc).to(ctx.device)).to_host()
    ref = of.permute(B.m, B.n, B.colptr, B.rowidx, B.vals, pr, pc)
    np.testing.assert_array_equal(got.colptr, ref[0])
    np.testing.assert_array_equal(got.rowidx, ref[1])
    np.testing.assert_array_equal(got.vals, ref[2])


def test_permute_rejects_non_permutations(ctx):
    import torch
    s = sp()
    A = gen.random_csc(50, 50, 0.1, 0x7301, PT_I64)
    dA = s.Matrix.from_host(ctx, A, PT_I64)
    dup = torch.zeros(50, dtype=torch.int32, device=ctx.device)
    out_of_range = torch.arange(50, dtype=torch.int32, device=ctx.device) + 1
    for bad in (dup, out_of_range):
        with pytest.raises(s.SpGEMMError):
            s.spgemm_mat_permute(ctx, dA, bad, None)
    ok = s.spgemm_mat_permute(ctx, dA, None, None).to_host()   # identity
    np.testing.assert_array_equal(ok.rowidx, A.rowidx)


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_summa_expand_sort_compress(ctx, sr):
    """Stage products by expand-sort-compress (the data-parallel outer-product
    multiply of Section 2.4) give the oracle's C, ragged grids and merge groups
    included."""
    for t, (m, k, n, d, g, every) in enumerate([(37, 29, 41, 0.1, 4, 0), (300, 200, 150, 0.03, 16, 0),
                                                (100, 64, 90, 0.05, 7, 3)]):
        A = gen.random_csc(m, k, d, 500 + t, sr)
        B = gen.random_csc(k, n, d, 600 + t, sr)
        C = blocked(ctx, A, B, sr, g, block_kernel=1, summa_merge_every=every)
        assert_matches(C, oracle.spgemm(A, B, sr), sr, what=f"{(m, k, n, g, every)}")
    A = gen.rmat(12, 8, 0x1216, sr)
    assert_matches(blocked(ctx, A, A, sr, 16, block_kernel=1), oracle.spgemm(A, A, sr), sr)


def test_summa_expand_sort_compress_matches_column_tiers_scale16(ctx):
    """Both stage-product kernels give identical C on R-MAT scale 16 (exact semiring)."""
    sr = PT_I64
    A = gen.rmat(16, 8, 0x1616, sr)
    C0 = blocked(ctx, A, A, sr, 16)
    C1 = blocked(ctx, A, A, sr, 16, block_kernel=1)
    np.testing.assert_array_equal(C0.colptr, C1.colptr)
    np.testing.assert_array_equal(C0.rowidx, C1.rowidx)
    np.testing.assert_array_equal(C0.vals, C1.vals)
    np.testing.assert_array_equal(np.diff(C0.colptr), oracle.symbolic(A, A))


def test_degenerate_inputs_on_the_newer_paths(ctx):
    """Empty operands, an empty grid row, 1 x 1 and g larger than the matrix, through
    the expand-sort-compress stage kernel, the permutation and the block work."""
    import torch
    s = sp()
    Z = CSC(9, 7, np.zeros(8, np.int64), np.zeros(0, np.int32), np.zeros(0))
    Y = CSC(7, 5, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0))
    C = blocked(ctx, Z, Y, PT_F64, 4, block_kernel=1)
    assert C.nnz == 0 and list(C.colptr) == [0] * 6
    one = CSC(1, 1, np.array([0, 1]), np.array([0], np.int32), np.array([3.0]))
    for kw in ({}, {"block_kernel": 1}):
        C = blocked(ctx, one, one, PT_F64, 4, **kw)    # g > dimension: 15 of 16 blocks empty
        assert C.nnz == 1 and C.vals[0] == 9.0
    # rows only in the first quarter: three block rows of A are empty
    A = gen.random_csc(40, 40, 0.1, 0x71, PT_I64)
    keep = A.rowidx < 10
    cp = np.concatenate([[0], np.cumsum([keep[A.colptr[j]:A.colptr[j + 1]].sum() for j in range(40)])])
    A = CSC(40, 40, cp.astype(np.int64), A.rowidx[keep], A.vals[keep])
    R = oracle.spgemm(A, A, PT_I64)
    for kw in ({}, {"block_kernel": 1}):
        assert_matches(blocked(ctx, A, A, PT_I64, 4, **kw), R, PT_I64, what=str(kw))
    dZ = s.Matrix.from_host(ctx, Z, PT_F64)
    assert s.spgemm_mat_permute(ctx, dZ, torch.arange(9, dtype=torch.int32, device=ctx.device).flip(0),
                                None).to_host().nnz == 0
    bf = s.spgemm_summa_block_flops(ctx, dZ, s.Matrix.from_host(ctx, Y, PT_F64), 3)
    assert bf.shape == (3, 3, 3) and bf.sum() == 0
