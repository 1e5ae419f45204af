"""Pins for the predictor-feature and network oracles, and generator checks."""
import math

import numpy as np

import oracle
from oracle import features as ofe
from oracle import mlp as om
from paper_1006_2183_gb300 import gen


def test_features_against_sets():
    A = gen.rmat(9, 8, 5)
    B = gen.erdos_renyi(512, 64, 4, 6)
    d, fl, mx, pc = ofe.raw_features(A, B)
    nnz = oracle.symbolic(A, B)
    for j in range(B.n):
        ks = B.rowidx[B.colptr[j]:B.colptr[j + 1]].tolist()
        sets = [set(A.rowidx[A.colptr[k]:A.colptr[k + 1]].tolist()) for k in ks]
        assert d[j] == len(ks)
        assert fl[j] == sum(len(s) for s in sets)
        assert mx[j] == max((len(s) for s in sets), default=0)
        union = set().union(*sets) if sets else set()
        assert nnz[j] == len(union)
        # the sketch of the union equals the OR of the per-column sketches
        bits = {int(b) for b in ofe.row_hash_bit(np.array(sorted(union), dtype=np.int64))} if union else set()
        assert pc[j] == len(bits)
        assert mx[j] <= nnz[j] <= min(fl[j], A.m)


def test_row_hash_bit_definition():
    i = np.array([0, 1, 2, 12345, 2 ** 31 - 1])
    want = [((int(v) * 0x9E3779B1) & 0xFFFFFFFF) >> 26 for v in i]
    np.testing.assert_array_equal(ofe.row_hash_bit(i), want)


def test_feature_vector_values():
    x = ofe.feature_vector([3], [10], [6], [0], 100)
    assert x.shape == (1, 8)
    np.testing.assert_allclose(x[0], [math.log1p(3), math.log1p(10), math.log1p(6), math.log1p(100), 0.0,
                                      math.log1p(10), math.log1p(4), 0.0])
    x = ofe.feature_vector([1], [1000], [1000], [64], 50)
    assert x[0, 5] == math.log1p(50)
    np.testing.assert_allclose(x[0, 4], math.log1p(64 * math.log(64 / 0.5)))


def test_mlp_gradient_finite_differences():
    rng = np.random.default_rng(0)
    theta = rng.normal(0, 0.3, om.NPARAM)
    X = rng.normal(0, 1, (13, 8))
    t = rng.normal(0, 1, 13)
    g = om.grad(theta, X, t)
    h = 1e-6
    for idx in rng.choice(om.NPARAM, 60, replace=False):
        e = np.zeros(om.NPARAM); e[idx] = h
        fd = (om.loss(theta + e, X, t) - om.loss(theta - e, X, t)) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, g[idx])


def test_mlp_closed_form_linear_case():
    # W1 = [I8; 0], b1 = 1 (so every unit is active for x >= 0), W2 = I, w3 = c, b3 = 0:
    # y = c . (x + 1) on the first 8 units
    theta = np.zeros(om.NPARAM)
    W1, b1, W2, b2, w3, b3 = om.unpack(theta)
    W1[:8, :8] = np.eye(8); b1[:] = 1.0
    W2[:, :] = np.eye(32)
    c = np.arange(1, 33, dtype=np.float64); w3[:] = c
    X = np.abs(np.random.default_rng(1).normal(size=(5, 8)))
    y, _ = om.forward(theta, X)
    want = (X + 1.0) @ c[:8] + c[8:].sum() * 1.0
    np.testing.assert_allclose(y, want)
    # the loss gradient wrt b3 is the mean of 2 (y - t)
    t = np.zeros(5)
    g = om.grad(theta, X, t)
    assert abs(g[-1] - np.mean(2 * y)) < 1e-9


def test_adam_first_step_moves_by_lr():
    theta = np.zeros(4); g = np.array([1.0, -2.0, 0.5, 0.0])
    th, m, v = om.adam_step(theta, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    np.testing.assert_allclose(th[:3], -0.01 * np.sign(g[:3]), rtol=1e-6)
    assert th[3] == 0


# ---------------------------------------------------------------- generators
def test_splitmix_reference_values():
    # SplitMix64 with state seeded at 0: first outputs of the published generator
    z = gen._mix(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF


def test_rmat_shape_and_dedup():
    A = gen.rmat(12, 8, 0x1802)
    assert A.m == A.n == 4096
    assert A.nnz <= 8 * 4096
    for j in range(0, A.n, 97):
        r = A.rowidx[A.colptr[j]:A.colptr[j + 1]]
        assert np.all(np.diff(r) > 0)
    B = gen.rmat(12, 8, 0x1802)
    np.testing.assert_array_equal(A.rowidx, B.rowidx)
    np.testing.assert_array_equal(A.vals, B.vals)
    # skew: column 0 (all bits 0) is the heaviest in expectation
    lens = np.diff(A.colptr)
    assert lens[0] >= np.percentile(lens, 99)


def test_rmat_non_power_of_two():
    A = gen.rmat(11, 4, 9, n=1500)
    assert A.m == A.n == 1500 and A.rowidx.max() < 1500


def test_er_exact_per_column():
    A = gen.erdos_renyi(4096, 4096, 8, 0x1001)
    assert np.all(np.diff(A.colptr) == 8)
    for j in range(0, 4096, 111):
        r = A.rowidx[A.colptr[j]:A.colptr[j + 1]]
        assert np.all(np.diff(r) > 0)


def test_frontier_counts():
    F = gen.frontier(1 << 14, 32, 3)
    lens = np.diff(F.colptr)
    assert lens.min() >= 1 and lens.max() <= 1000


def test_batch_pairs_shapes():
    pairs = gen.batch_pairs(6, 0x4004, 6, 9)
    for A, B in pairs:
        assert A.n == B.m and 64 <= A.n < 512
        assert A.vals.dtype == np.int64 and A.vals.min() >= -8 and A.vals.max() <= 8


def test_generators_do_not_depend_on_threads(monkeypatch):
    """Threaded generation fills chunks of counters; the matrices must not depend on
    the chunking or on whether threads are used."""
    ref = gen.rmat(12, 8, 0x77)
    refp = gen.batch_pairs(3, 0x99, 6, 9)
    monkeypatch.setattr(gen, "_EDGE_CHUNK", 1000)
    thr = gen.rmat(12, 8, 0x77)
    gen._tls.serial = True
    try:
        ser = gen.rmat(12, 8, 0x77)
    finally:
        gen._tls.serial = False
    for M in (thr, ser):
        np.testing.assert_array_equal(M.colptr, ref.colptr)
        np.testing.assert_array_equal(M.rowidx, ref.rowidx)
        np.testing.assert_array_equal(M.vals, ref.vals)
    for (a, b), (c, d) in zip(gen.batch_pairs(3, 0x99, 6, 9), refp):
        np.testing.assert_array_equal(a.rowidx, c.rowidx)
        np.testing.assert_array_equal(b.vals, d.vals)


def test_restriction_shape():
    for n, order in ((1000, 2), (1000, 4), (1003, 8)):
        S = gen.restriction(n, order, 0x88)
        assert S.m == -(-n // order) and S.n == n and S.nnz == n
        sizes = np.bincount(S.rowidx, minlength=S.m)
        assert np.all(sizes[:-1] == order) and 1 <= sizes[-1] <= order
