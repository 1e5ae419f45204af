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


def test_summa_scale18_sampled(ctx):
    """The benchmark's blocked workload: R-MAT scale 18 on a 16 x 16 grid, PT64;
    column counts vs the oracle's symbolic pass and sampled columns vs the oracle."""
    sr = PT_F64
    A = gen.rmat(18, 8, 0x1802, sr)
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
        assert np.all(np.abs(got - ref) <= 1e-13 * np.abs(ref)), j
