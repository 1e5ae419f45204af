"""Full-size parity for the larger workloads, checked against the oracle where it can
run and against closed forms where the result has one:

* the multigrid Galerkin product R*A*P on a 128^3 grid (7-point Laplacian, 2x2x2
  aggregation), plain and with the learned predictor plus autotuned bins, equal to
  the coarse 7-point operator with diagonal 24 and couplings -4, bit for bit;
* 512 uneven int64 pairs in one batch, plain and learned+batched: every column count
  against the oracle's symbolic pass, sampled columns against the oracle, and the two
  forms identical;
* the tall-skinny BFS step, boolean R-MAT scale 20 (edge factor 16) times a 2^20 x 128
  frontier, every column against the oracle;
* R-MAT scale 20 A*A (edge factor 8), plus-times FP64 and or-and, flat, on a
  32 x 32 virtual SUMMA grid and flat with the learned predictor: every column count
  against the oracle, sampled columns against the oracle, and the three structures
  identical (boolean values too).
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_sampled, device_columns, sp
from helpers import OR_BOOL, PT_F64, PT_I64
from paper_1006_2183_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return sp().Context(stream=torch.cuda.Stream())


def _release():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _train_predictor(ctx, steps=300):
    """A predictor trained on exact symbolic counts of small R-MAT and ER squares drawn
    from seeds disjoint from every workload below."""
    s = sp()
    Xs, ys = [], []
    for M in (gen.rmat(14, 8, 0x7000), gen.erdos_renyi(8192, 8192, 8, 0x7100), gen.rmat(15, 4, 0x7200)):
        d = s.Matrix.from_host(ctx, M, PT_F64)
        X, y = s.spgemm_predictor_features(ctx, d, d)
        keep = y > 0
        Xs.append(X[keep])
        ys.append(torch.log1p(y[keep].double()).float())
    X, y = torch.cat(Xs), torch.cat(ys)
    s.spgemm_predictor_set(ctx, np.random.default_rng(11).normal(0, 0.2, s.NPARAM).astype(np.float32))
    for _ in range(steps):
        s.spgemm_predictor_train_step(ctx, X, y, 3e-3)


def _checksums(C, chunk=1 << 27):
    """Order-sensitive int64 fingerprints of a device result (colptr, rows, values),
    summed modulo 2^64 in chunks so that no large temporary is made."""
    m, n, nnz, cp, ir, v = C.export()
    torch.cuda.current_stream().wait_stream(C.ctx.stream)
    hc = int((cp * (torch.arange(n + 1, device=cp.device) % 997 + 1)).sum())
    hr = hv = 0
    for lo in range(0, nnz, chunk):
        hi = min(lo + chunk, nnz)
        w = torch.arange(lo, hi, device=ir.device, dtype=torch.int64) % 1000003 + 1
        vv = v[lo:hi].view(torch.int64) if v.dtype == torch.float64 else v[lo:hi].to(torch.int64)
        hr = (hr + int((ir[lo:hi].to(torch.int64) * w).sum())) % (1 << 64)
        hv = (hv + int((vv * w).sum())) % (1 << 64)
    return n, nnz, hc, hr, hv


def test_galerkin_128_plain_and_learned(ctx):
    s = sp()
    N = 128
    A = gen.grid3d_laplacian(N)
    P = gen.aggregation_2x2x2(N)
    R = gen.transpose_host(P)
    coarse = gen.grid3d_laplacian(N // 2)
    dA, dP, dR = (s.Matrix.from_host(ctx, M, PT_F64) for M in (A, P, R))
    _train_predictor(ctx)
    tuned = s.spgemm_autotune(ctx, [dA], [dP], PT_F64)
    learned = s.default_opts(use_predictor=1, warp_max_flops=tuned.warp_max_flops,
                             block_max_flops=tuned.block_max_flops, dense_part_flops=tuned.dense_part_flops)
    for label, opts in (("plain", None), ("learned", learned)):
        AP = s.spgemm_batch(ctx, [dA], [dP], PT_F64, opts)[0]
        assert AP.export()[2] == 32 * 64 ** 3 - 24 * 64 ** 2, label
        RAP = s.spgemm_batch(ctx, [dR], [AP], PT_F64, opts)[0].to_host()
        np.testing.assert_array_equal(RAP.colptr, coarse.colptr, err_msg=label)
        np.testing.assert_array_equal(RAP.rowidx, coarse.rowidx, err_msg=label)
        np.testing.assert_array_equal(RAP.vals, 4.0 * coarse.vals, err_msg=label)
        del AP, RAP
    _release()


def test_batch_512_uneven_pairs_plain_and_learned(ctx):
    s = sp()
    pairs = gen.batch_pairs(512, 0x4004)
    As = [s.Matrix.from_host(ctx, a, PT_I64) for a, _ in pairs]
    Bs = [s.Matrix.from_host(ctx, b, PT_I64) for _, b in pairs]
    rng = np.random.default_rng(0x4004)
    Cs = s.spgemm_batch(ctx, As, Bs, PT_I64)
    sums = []
    for i, ((a, b), C) in enumerate(zip(pairs, Cs)):
        lens = np.diff(b.colptr)
        cols = np.unique(np.concatenate([rng.choice(b.n, 4, replace=False), [int(np.argmax(lens))]]))
        cp = assert_sampled(C, a, b, PT_I64, cols, what=f"pair {i}")
        np.testing.assert_array_equal(np.diff(cp), oracle.symbolic(a, b), err_msg=f"pair {i} counts")
        sums.append(_checksums(C))
    del Cs
    _release()
    _train_predictor(ctx, steps=200)
    tuned = s.spgemm_autotune(ctx, As[:64], Bs[:64], PT_I64)
    opts = s.default_opts(use_predictor=1, warp_max_flops=tuned.warp_max_flops,
                          block_max_flops=tuned.block_max_flops, dense_part_flops=tuned.dense_part_flops)
    Cs = s.spgemm_batch(ctx, As, Bs, PT_I64, opts)
    for i, C in enumerate(Cs):
        assert _checksums(C) == sums[i], f"pair {i}: learned+batched differs from plain"
    del Cs
    _release()


def test_bfs_step_rmat20_frontier(ctx):
    s = sp()
    A = gen.rmat(20, 16, 0x4F00, OR_BOOL)
    F = gen.frontier(A.m, 128, 0x4F01, 1, 1000)
    C = s.spgemm_batch(ctx, [s.Matrix.from_host(ctx, A, OR_BOOL)], [s.Matrix.from_host(ctx, F, OR_BOOL)],
                       OR_BOOL)[0]
    assert_sampled(C, A, F, OR_BOOL, np.arange(F.n), what="bfs")
    del C
    _release()


@pytest.mark.parametrize("sr", [PT_F64, OR_BOOL])
def test_rmat20_flat_and_summa32(ctx, sr):
    s = sp()
    A = gen.rmat(20, 8, 0x2005, sr)
    counts = oracle.symbolic(A, A)
    dA = s.Matrix.from_host(ctx, A, sr)
    lens = np.diff(A.colptr)
    rng = np.random.default_rng(0x2005)
    cols = np.unique(np.concatenate([np.argsort(lens)[-8:], rng.choice(A.n, 120, replace=False)]))
    C = s.spgemm_multiply(ctx, dA, dA, sr)
    cp = assert_sampled(C, A, A, sr, cols, what="flat")
    np.testing.assert_array_equal(np.diff(cp), counts)
    fl = _checksums(C)
    flat_rows, flat_vals = fl[:4], fl[4]
    del C
    _release()
    C = s.spgemm_summa_blocked(ctx, dA, dA, 32, sr)
    cp = assert_sampled(C, A, A, sr, cols, what="summa 32")
    np.testing.assert_array_equal(np.diff(cp), counts)
    assert _checksums(C)[:4] == flat_rows, "flat and blocked structure differ"
    del C
    _release()
    # the large skewed squaring with the learned predictor sizing the output (trained on
    # R-MAT scales 14-15 and ER 2^13 here; every overflowed column is redone exactly): the same counts,
    # sampled columns and structure as the exact path, values exact for the boolean semiring
    _train_predictor(ctx, steps=200)
    C = s.spgemm_multiply(ctx, dA, dA, sr, s.default_opts(use_predictor=1))
    cp = assert_sampled(C, A, A, sr, cols, what="flat, predictor on")
    np.testing.assert_array_equal(np.diff(cp), counts)
    got = _checksums(C)
    assert got[:4] == flat_rows, "predicted and exact structure differ"
    if sr == OR_BOOL:
        assert got[4] == flat_vals, "predicted and exact boolean values differ"
    del C
    _release()
