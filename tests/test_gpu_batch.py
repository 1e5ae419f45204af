"""Batched products (one item space, persistent tier launches), batch plans replayed
from a CUDA graph with new values, autotuned thresholds, and the Galerkin triple
product R*A*P -- all against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_matches, sp
from helpers import OR_BOOL, PT_F64, PT_I64
from paper_1006_2183_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    s = sp()
    return s.Context(stream=torch.cuda.Stream())   # a capturable stream


def _up(ctx, M, sr):
    return sp().Matrix.from_host(ctx, M, sr)


def test_batch_uneven_pairs_int64(ctx):
    s = sp()
    pairs = gen.batch_pairs(24, 0x4004, 6, 11)
    As = [_up(ctx, a, PT_I64) for a, _ in pairs]
    Bs = [_up(ctx, b, PT_I64) for _, b in pairs]
    Cs = s.spgemm_batch(ctx, As, Bs, PT_I64)
    for (a, b), C in zip(pairs, Cs):
        assert_matches(C.to_host(), oracle.spgemm(a, b, PT_I64), PT_I64)


def test_batch_equals_individual_and_mixed_sizes(ctx):
    s = sp()
    mats = [gen.rmat(12, 8, 1), gen.erdos_renyi(300, 300, 3, 2), gen.rmat(9, 16, 3), gen.erdos_renyi(50, 50, 40, 4)]
    As = [_up(ctx, M, PT_F64) for M in mats]
    Cs = s.spgemm_batch(ctx, As, As, PT_F64)
    for M, C in zip(mats, Cs):
        assert_matches(C.to_host(), oracle.spgemm(M, M, PT_F64), PT_F64)


def test_batch_bool_bfs_step(ctx):
    """Tall-skinny BFS step A (x) F over (or, and) as a batch of one."""
    s = sp()
    A = gen.rmat(14, 16, 0x4F00, OR_BOOL)
    F = gen.frontier(A.m, 128, 0x4F01, 1, 1000)
    C = s.spgemm_batch(ctx, [_up(ctx, A, OR_BOOL)], [_up(ctx, F, OR_BOOL)], OR_BOOL)[0]
    assert_matches(C.to_host(), oracle.spgemm(A, F, OR_BOOL), OR_BOOL)


def test_batch_plan_graph_replay_new_values(ctx):
    s = sp()
    pairs = gen.batch_pairs(10, 0x4104, 7, 10)
    dev = ctx.device
    vals = []
    As, Bs = [], []
    for a, b in pairs:
        va = torch.from_numpy(a.vals.copy()).to(dev)
        vb = torch.from_numpy(b.vals.copy()).to(dev)
        vals.append((va, vb))
        As.append(s.Matrix.csc(ctx, a.m, a.n, torch.from_numpy(a.colptr).to(dev), torch.from_numpy(a.rowidx).to(dev),
                               va, PT_I64))
        Bs.append(s.Matrix.csc(ctx, b.m, b.n, torch.from_numpy(b.colptr).to(dev), torch.from_numpy(b.rowidx).to(dev),
                               vb, PT_I64))
    plan = s.spgemm_batch_plan(ctx, As, Bs, PT_I64)
    outs = plan.outputs()
    for rnd in range(3):
        if rnd:
            with torch.cuda.stream(ctx.stream):
                for va, vb in vals:
                    va.mul_(-1).add_(rnd)
                    vb.add_(2 * rnd)
        plan.execute()   # first call: eager run + capture; later calls: graph replay
        ctx.stream.synchronize()
        for (a, b), (va, vb), C in zip(pairs, vals, outs):
            a2 = a.with_vals(va.cpu().numpy())
            b2 = b.with_vals(vb.cpu().numpy())
            assert_matches(C.to_host(), oracle.spgemm(a2, b2, PT_I64), PT_I64, what=f"round {rnd}")


def test_autotune_keeps_results(ctx):
    s = sp()
    pairs = gen.batch_pairs(8, 0x4204, 8, 11)
    As = [_up(ctx, a, PT_I64) for a, _ in pairs]
    Bs = [_up(ctx, b, PT_I64) for _, b in pairs]
    o = s.spgemm_autotune(ctx, As, Bs, PT_I64)
    assert o.warp_max_flops in (128, 512) and o.block_max_flops in (1024, 4096)
    Cs = s.spgemm_batch(ctx, As, Bs, PT_I64, o)
    for (a, b), C in zip(pairs, Cs):
        assert_matches(C.to_host(), oracle.spgemm(a, b, PT_I64), PT_I64)


@pytest.mark.parametrize("N", [8, 32])
def test_galerkin_triple_product(ctx, N):
    """R*A*P with the 7-point Laplacian and 2x2x2 aggregation equals the coarse
    7-point operator with diagonal 24 and couplings -4 (exact in FP64)."""
    s = sp()
    A = gen.grid3d_laplacian(N)
    P = gen.aggregation_2x2x2(N)
    R = gen.transpose_host(P)
    dA, dP, dR = _up(ctx, A, PT_F64), _up(ctx, P, PT_F64), _up(ctx, R, PT_F64)
    AP = s.spgemm_batch(ctx, [dA], [dP], PT_F64)[0]
    RAP = s.spgemm_batch(ctx, [dR], [AP], PT_F64)[0].to_host()
    coarse = gen.grid3d_laplacian(N // 2)
    np.testing.assert_array_equal(RAP.colptr, coarse.colptr)
    np.testing.assert_array_equal(RAP.rowidx, coarse.rowidx)
    np.testing.assert_array_equal(RAP.vals, 4.0 * coarse.vals)


def test_autotuned_batch_is_never_slower_than_either_predictor_choice(ctx):
    """The autotuner times whole batched calls with and without the learned predictor
    and keeps the faster: the tuned call is no slower (beyond timing noise) than either
    fixed choice at the same thresholds, and its output equals the exact path's."""
    import time
    import torch
    s = sp()
    pairs = gen.batch_pairs(96, 0x4104, 9, 13)
    As = [_up(ctx, a, PT_I64) for a, _ in pairs]
    Bs = [_up(ctx, b, PT_I64) for _, b in pairs]
    rng = np.random.default_rng(5)
    s.spgemm_predictor_set(ctx, rng.normal(0, 0.2, s.NPARAM).astype(np.float32))
    tuned = s.spgemm_autotune(ctx, As, Bs, PT_I64, s.default_opts(use_predictor=1))
    thr = dict(warp_max_flops=tuned.warp_max_flops, block_max_flops=tuned.block_max_flops,
               dense_part_flops=tuned.dense_part_flops)

    def best_of(opts, reps=7):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            Cs = s.spgemm_batch(ctx, As, Bs, PT_I64, opts)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
            del Cs
        return min(ts)
    t_auto = best_of(tuned)
    t_on = best_of(s.default_opts(use_predictor=1, **thr))
    t_off = best_of(s.default_opts(use_predictor=0, **thr))
    assert t_auto <= 1.25 * min(t_on, t_off), (t_auto, t_on, t_off, tuned.use_predictor)
    ref = [C.to_host() for C in s.spgemm_batch(ctx, As, Bs, PT_I64, s.default_opts(use_predictor=0, **thr))]
    for C, R in zip(s.spgemm_batch(ctx, As, Bs, PT_I64, tuned), ref):
        H = C.to_host()
        np.testing.assert_array_equal(H.colptr, R.colptr)
        np.testing.assert_array_equal(H.rowidx, R.rowidx)
        np.testing.assert_array_equal(H.vals, R.vals)
