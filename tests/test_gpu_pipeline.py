"""Parity of the two-stream SUMMA pipeline (stage merges on a second stream,
overlapping the next group's stage products; Sections 7.2-7.3) with the oracle
and with the one-stream blocked product.

The pipeline runs the same merges in the same order as spgemm_summa_blocked with
the same summa_merge_every, so structure and the exact semirings must match the
oracle bit for bit, plus-times FP64 within 1e-13 relative.
"""
import numpy as np
import pytest

import oracle
from gpu_util import assert_matches, assert_sampled, sp
from helpers import MP_F32, OR_BOOL, PT_F64, PT_I64
from paper_1006_2183_gb300 import gen
from paper_1006_2183_gb300.gen import CSC

pytestmark = pytest.mark.gpu
SEMIRINGS = [PT_F64, MP_F32, OR_BOOL, PT_I64]


@pytest.fixture(scope="module")
def ctxs():
    import torch
    s = sp()
    return s.Context(), s.Context(stream=torch.cuda.Stream())


def pipelined(ctxs, A, B, sr, g, **kw):
    s = sp()
    ctx, mctx = ctxs
    dA = s.Matrix.from_host(ctx, A, sr)
    dB = dA if B is A else s.Matrix.from_host(ctx, B, sr)
    return s.spgemm_summa_pipelined(ctx, mctx, dA, dB, g, sr, s.default_opts(**kw) if kw else None)


@pytest.mark.parametrize("sr", SEMIRINGS)
@pytest.mark.parametrize("every", [1, 2, 3, 8])
def test_pipeline_rmat_matches_oracle(ctxs, sr, every):
    A = gen.rmat(11, 8, 0x1108, sr)
    R = oracle.spgemm(A, A, sr)
    C = pipelined(ctxs, A, A, sr, 8, summa_merge_every=every)
    assert C.ctx is ctxs[1]
    assert_matches(C.to_host(), R, sr, what=f"every {every}")


@pytest.mark.parametrize("sr", [PT_I64, MP_F32])
def test_pipeline_rectangular_ragged(ctxs, sr):
    for t, (m, k, n, d, g, every) in enumerate([(37, 29, 41, 0.1, 4, 1), (100, 64, 90, 0.05, 7, 2),
                                                (5, 3, 2, 0.6, 4, 1), (300, 200, 150, 0.03, 16, 5),
                                                (1, 20, 30, 0.3, 3, 1)]):
        A = gen.random_csc(m, k, d, 500 + t, sr)
        B = gen.random_csc(k, n, d, 600 + t, sr)
        R = oracle.spgemm(A, B, sr)
        assert_matches(pipelined(ctxs, A, B, sr, g, summa_merge_every=every).to_host(), R, sr,
                       what=f"{(m, k, n, g, every)}")


def test_pipeline_equals_one_stream(ctxs):
    """Same merges in the same order: identical to spgemm_summa_blocked, and the same stage statistics."""
    s = sp()
    ctx, _ = ctxs
    sr = PT_I64
    A = gen.rmat(13, 8, 0x1313, sr)
    dA = s.Matrix.from_host(ctx, A, sr)
    o = s.default_opts(summa_merge_every=2)
    Cb = s.spgemm_summa_blocked(ctx, dA, dA, 8, sr, o).to_host()
    stats_b = s.spgemm_summa_stats(ctx, 8)
    Cp = s.spgemm_summa_pipelined(ctx, ctxs[1], dA, dA, 8, sr, o).to_host()
    stats_p = s.spgemm_summa_stats(ctx, 8)
    np.testing.assert_array_equal(Cp.colptr, Cb.colptr)
    np.testing.assert_array_equal(Cp.rowidx, Cb.rowidx)
    np.testing.assert_array_equal(Cp.vals, Cb.vals)
    assert stats_p == stats_b
    assert sum(stats_p[0]) == int(oracle.flops_per_col(A, A).sum())


def test_pipeline_empty_groups_and_errors(ctxs):
    s = sp()
    ctx, mctx = ctxs
    # no nonzeros at all: every group is empty
    Z = CSC(9, 7, np.zeros(8, np.int64), np.zeros(0, np.int32), np.zeros(0))
    Y = CSC(7, 5, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0))
    C = pipelined(ctxs, Z, Y, PT_F64, 4, summa_merge_every=1).to_host()
    assert C.nnz == 0 and list(C.colptr) == [0] * 6
    # inner dimension 3 on a 6 x 6 grid: stages 3..5 hold no blocks
    A = gen.random_csc(20, 3, 0.5, 7, PT_I64)
    B = gen.random_csc(3, 20, 0.5, 8, PT_I64)
    assert_matches(pipelined(ctxs, A, B, PT_I64, 6, summa_merge_every=1).to_host(), oracle.spgemm(A, B, PT_I64),
                   PT_I64, what="empty stages")
    dA = s.Matrix.from_host(ctx, A, PT_I64)
    dB = s.Matrix.from_host(ctx, B, PT_I64)
    with pytest.raises(s.SpGEMMError):
        s.spgemm_summa_pipelined(ctx, ctx, dA, dB, 4, PT_I64)        # one context for both streams
    with pytest.raises(s.SpGEMMError):
        s.spgemm_summa_pipelined(ctx, mctx, dA, dA, 4, PT_I64)       # 20 x 3 times 20 x 3
    with pytest.raises(s.SpGEMMError):
        s.spgemm_summa_pipelined(ctx, mctx, dA, dB, 0, PT_I64)       # g = 0
    # both contexts still work after the errors
    assert_matches(s.spgemm_summa_pipelined(ctx, mctx, dA, dB, 4, PT_I64,
                                            s.default_opts(summa_merge_every=1)).to_host(),
                   oracle.spgemm(A, B, PT_I64), PT_I64, what="after errors")


def test_pipeline_stream_ordered_allocator_and_repeats(ctxs):
    """Merge context on the library's stream-ordered allocator; repeated calls free what they take."""
    import torch
    s = sp()
    ctx, _ = ctxs
    mctx = s.Context(stream=torch.cuda.Stream(), torch_allocator=False)
    sr = MP_F32
    A = gen.rmat(10, 8, 0x1010, sr)
    R = oracle.spgemm(A, A, sr)
    dA = s.Matrix.from_host(ctx, A, sr)
    o = s.default_opts(summa_merge_every=1)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    for _ in range(5):
        C = s.spgemm_summa_pipelined(ctx, mctx, dA, dA, 4, sr, o)
        assert_matches(C.to_host(), R, sr, what="repeat")
        del C
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_pipeline_scale16_grid16(ctxs):
    """R-MAT scale 16 on a 16 x 16 grid, merges every 4 stages: the whole structure
    equals the one-stream product and sampled columns match the oracle."""
    s = sp()
    ctx, mctx = ctxs
    sr = PT_F64
    A = gen.rmat(16, 8, 0x1602, sr)
    dA = s.Matrix.from_host(ctx, A, sr)
    o = s.default_opts(summa_merge_every=4)
    Cp = s.spgemm_summa_pipelined(ctx, mctx, dA, dA, 16, sr, o)
    cols = np.random.default_rng(16).choice(A.n, 256, replace=False)
    cols.sort()
    assert_sampled(Cp, A, A, sr, cols, what="scale 16 pipelined")
    Hp = Cp.to_host()
    Hb = s.spgemm_summa_blocked(ctx, dA, dA, 16, sr, o).to_host()
    np.testing.assert_array_equal(Hp.colptr, Hb.colptr)
    np.testing.assert_array_equal(Hp.rowidx, Hb.rowidx)
    np.testing.assert_allclose(Hp.vals, Hb.vals, rtol=2e-13, atol=0)


@pytest.mark.parametrize("sr", [PT_I64, OR_BOOL])
def test_pipeline_with_expand_sort_compress_stages(ctxs, sr):
    """Stage products in the outer-product order (block_kernel = 1) feeding the
    pipelined merges: the same C as the oracle."""
    A = gen.rmat(11, 8, 0x110E, sr)
    R = oracle.spgemm(A, A, sr)
    for every in (1, 3):
        C = pipelined(ctxs, A, A, sr, 8, summa_merge_every=every, block_kernel=1)
        assert_matches(C.to_host(), R, sr, what=f"esc, every {every}")


def test_pipeline_single_group_upper_bound_slots(ctxs):
    """One group (merge after the last stage): its partials go to upper-bound slots
    and the worker's single merge reads them with gaps."""
    sr = MP_F32
    A = gen.rmat(13, 8, 0x1313, sr)
    R = oracle.spgemm(A, A, sr)
    assert_matches(pipelined(ctxs, A, A, sr, 16).to_host(), R, sr, what="single group")
