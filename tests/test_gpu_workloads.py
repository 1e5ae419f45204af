"""Second workloads on the same kernels (Section 6.2): multiplication with the
restriction operator of a graph contraction, A S^T and S A S^T, of orders 2, 4
and 8 (Section 6.2.3), and R-MAT times tall-skinny Erdos-Renyi right-hand sides
whose nonzeros per column sweep 1 .. 10^4 (Section 6.2.2) -- against the oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_matches, assert_sampled, sp
from helpers import PT_F64, PT_I64
from paper_1006_2183_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return sp().Context()


@pytest.mark.parametrize("order", [2, 4, 8])
@pytest.mark.parametrize("sr", [PT_F64, PT_I64])
def test_restriction_products(ctx, sr, order):
    """A S^T and the contraction S A S^T: whole results against the oracle; in int64
    the contraction keeps the total edge weight (every edge lands in one aggregate pair)."""
    s = sp()
    A = gen.rmat(14, 8, 0x6201, sr)
    S = gen.restriction(A.n, order, 0x6202 + order, sr)
    St = gen.transpose_host(S)
    dA, dS, dSt = (s.Matrix.from_host(ctx, M, sr) for M in (A, S, St))
    ASt = s.spgemm_multiply(ctx, dA, dSt, sr)
    ref = oracle.spgemm(A, St, sr)
    assert_matches(ASt.to_host(), ref, sr, what=f"A S^T order {order}")
    SASt = s.spgemm_multiply(ctx, dS, ASt, sr).to_host()
    ref2 = oracle.spgemm(S, ref, sr)
    assert_matches(SASt, ref2, sr, what=f"S A S^T order {order}")
    assert SASt.m == SASt.n == -(-A.n // order)
    if sr == PT_I64:
        assert int(SASt.vals.sum()) == int(A.vals.sum())


@pytest.mark.parametrize("c2", [1, 10, 100, 1000, 10000])
def test_tall_skinny_sweep(ctx, c2):
    """R-MAT (8 per column) times an n x k Erdos-Renyi matrix with c2 nonzeros per
    column, k = n / 2^13 as in the paper's scaled runs (n/p = 2^14, k/p = 2)."""
    s = sp()
    A = gen.rmat(16, 8, 0x6301, PT_F64)
    k = A.n >> 13
    F = gen.erdos_renyi(A.n, k, c2, 0x6302 + c2, PT_F64)
    C = s.spgemm_multiply(ctx, s.Matrix.from_host(ctx, A, PT_F64), s.Matrix.from_host(ctx, F, PT_F64), PT_F64)
    cp = assert_sampled(C, A, F, PT_F64, np.arange(k), what=f"c2 = {c2}")
    np.testing.assert_array_equal(np.diff(cp), oracle.symbolic(A, F))
