"""Learned nnz predictor: device features vs the oracle's definitions, device
gradients vs the float64 oracle backprop, and products with the predictor on
that stay identical to the oracle (overflow repair included)."""
import numpy as np
import pytest

import oracle
from oracle import features as ofe
from oracle import mlp as om
from gpu_util import assert_matches, sp
from helpers import MP_F32, OR_BOOL, PT_F64, PT_I64
from paper_1006_2183_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return sp().Context()


def _theta(seed, scale=0.3):
    return np.random.default_rng(seed).normal(0, scale, om.NPARAM)


def test_features_match_oracle(ctx):
    s = sp()
    import torch
    A = gen.rmat(10, 8, 5)
    B = gen.erdos_renyi(1024, 200, 5, 6)
    dA, dB = s.Matrix.from_host(ctx, A, PT_F64), s.Matrix.from_host(ctx, B, PT_F64)
    X, y = s.spgemm_predictor_features(ctx, dA, dB)
    d, fl, mx, pc = ofe.raw_features(A, B)
    ref = ofe.feature_vector(d, fl, mx, pc, A.m)
    np.testing.assert_allclose(X.cpu().numpy(), ref, rtol=2e-6, atol=2e-6)
    np.testing.assert_array_equal(y.cpu().numpy(), oracle.symbolic(A, B))


def test_forward_and_gradient_match_float64_backprop(ctx):
    s = sp()
    import torch
    rng = np.random.default_rng(7)
    theta = _theta(1).astype(np.float32)
    X = rng.normal(0, 1, (777, 8)).astype(np.float32)
    t = rng.normal(0, 1, 777).astype(np.float32)
    s.spgemm_predictor_set(ctx, theta)
    dX = torch.from_numpy(X).to(ctx.device)
    out = s.spgemm_predictor_forward(ctx, dX).cpu().numpy()
    ref, _ = om.forward(theta.astype(np.float64), X.astype(np.float64))
    np.testing.assert_allclose(out, ref, rtol=1e-4, atol=1e-4)
    loss, g = s.spgemm_predictor_train_step(ctx, dX, torch.from_numpy(t).to(ctx.device), 1e-3, want_grad=True)
    gref = om.grad(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    lref = om.loss(theta.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lref) <= 1e-4 * max(1.0, lref)
    scale = np.max(np.abs(gref))
    np.testing.assert_allclose(g, gref, rtol=1e-3, atol=1e-4 * scale)
    # the step moved every parameter with a nonzero gradient by about lr (first Adam step)
    th2 = s.spgemm_predictor_get(ctx)
    moved = np.abs(th2 - theta)
    nz = np.abs(gref) > 1e-3 * scale
    assert np.all(np.abs(moved[nz] - 1e-3) < 2e-4)


def _pred_product(ctx, A, B, sr, theta):
    s = sp()
    s.spgemm_predictor_set(ctx, theta.astype(np.float32))
    dA = s.Matrix.from_host(ctx, A, sr)
    dB = dA if B is A else s.Matrix.from_host(ctx, B, sr)
    plan = s.spgemm_plan(ctx, dA, dB, sr, s.default_opts(use_predictor=1))
    C = s.spgemm_numeric(plan).to_host()
    return C, plan.stats()


@pytest.mark.parametrize("sr", [PT_F64, MP_F32, OR_BOOL, PT_I64])
def test_predictor_output_identical_under_underprediction(ctx, sr):
    """All-zero network: y = 0 -> capacity max(2, max len): most columns overflow and are repaired."""
    A = gen.rmat(12, 8, 0x5151, sr)
    R = oracle.spgemm(A, A, sr)
    C, st = _pred_product(ctx, A, A, sr, np.zeros(om.NPARAM))
    assert_matches(C, R, sr)
    assert st["overflow_cols"] > 0


def test_predictor_output_identical_under_overprediction(ctx):
    theta = np.zeros(om.NPARAM)
    theta[-1] = 30.0    # b3: predicts far above the bound, capacity = min(flops, m)
    A = gen.rmat(12, 8, 0x5252, PT_I64)
    C, st = _pred_product(ctx, A, A, PT_I64, theta)
    assert_matches(C, oracle.spgemm(A, A, PT_I64), PT_I64)
    assert st["overflow_cols"] == 0


def test_training_gains_over_the_bound(ctx):
    """Trained on symbolic-pass labels of R-MAT/ER matrices from disjoint seeds, the
    predictor's capacities are much tighter than the exact upper bound min(flops, m)
    that the method without it would have to allocate, with few overflows."""
    s = sp()
    import torch
    Xs, ys = [], []
    for i, mk in enumerate([lambda q: gen.rmat(11, 8, 0x7000 + q), lambda q: gen.erdos_renyi(2048, 2048, 6, 0x7100 + q),
                            lambda q: gen.rmat(12, 4, 0x7200 + q), lambda q: gen.rmat(10, 16, 0x7300 + q)]):
        for q in range(2):
            M = mk(q)
            d = s.Matrix.from_host(ctx, M, PT_F64)
            X, y = s.spgemm_predictor_features(ctx, d, d)
            keep = y > 0
            Xs.append(X[keep])
            ys.append(torch.log1p(y[keep].double()).float())
    X = torch.cat(Xs)
    y = torch.cat(ys)
    s.spgemm_predictor_set(ctx, _theta(3, 0.2).astype(np.float32))
    losses = []
    for it in range(400):
        loss, _ = s.spgemm_predictor_train_step(ctx, X, y, 3e-3)
        losses.append(loss)
    assert losses[-1] < 0.2 * losses[0]
    # evaluate on an unseen matrix
    A = gen.rmat(12, 8, 0x1234)
    fl = oracle.flops_per_col(A, A)
    nz = oracle.symbolic(A, A)
    theta = s.spgemm_predictor_get(ctx)
    C, st = _pred_product(ctx, A, A, PT_F64, theta)
    assert_matches(C, oracle.spgemm(A, A, PT_F64), PT_F64)
    dA = s.Matrix.from_host(ctx, A, PT_F64)
    Xe, _ = s.spgemm_predictor_features(ctx, dA, dA, want_labels=False)
    pred = np.expm1(s.spgemm_predictor_forward(ctx, Xe).cpu().numpy().astype(np.float64))
    bound = np.minimum(fl, A.m)
    cap = np.clip(np.ceil(1.25 * np.maximum(pred, 0)) + 2, 0, bound)
    gain = bound.sum() / max(cap.sum(), 1)
    assert gain > 1.3, gain
    assert st["overflow_cols"] < 0.15 * (nz > 0).sum()
