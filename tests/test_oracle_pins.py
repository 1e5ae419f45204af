"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test here checks the oracle against something other than itself: the
paper's worked examples (tests/golden/), closed forms, textbook special cases
computed by a different route, the inner-product definition (Eq. 1) by brute
force, and algebraic invariants.
"""
import numpy as np
import pytest

import oracle
from oracle import formats as of
from paper_1006_2183_gb300 import gen
from paper_1006_2183_gb300.gen import CSC

from helpers import (DT, FP64_RTOL, MP_F32, OR_BOOL, PT_F64, PT_I64, assert_csc_equal, assert_sorted_unique,
                     csc_to_dict, dense_bruteforce, pattern_matrix, read_golden)

SEMIRINGS = [PT_F64, MP_F32, OR_BOOL, PT_I64]


def _ints(line):
    return [int(x) for x in line.split()[1:]]


# ---------------------------------------------------------------- Figs. 5-7
def test_dcsc_nine_by_nine_example():
    g = {ln.split()[0]: ln.split()[1:] for ln in read_golden("fig5_fig6_9x9.txt")}
    m, n = int(g["m"][0]), int(g["n"][0])
    I = np.array([int(x) - 1 for x in g["triples_I"]])
    J = np.array([int(x) - 1 for x in g["triples_J"]])
    V = np.array([float(x) for x in g["triples_V"]])
    colptr, rowidx = gen.csc_from_coo(m, n, I, J)
    order = np.lexsort((I, J))
    # CSC of Fig. 5
    np.testing.assert_array_equal(colptr + 1, [int(x) for x in g["csc_JC"]])
    np.testing.assert_array_equal(rowidx + 1, [int(x) for x in g["csc_IR"]])
    np.testing.assert_allclose(V[order], [float(x) for x in g["csc_NUM"]])
    jc, cp, aux, chunk = of.to_dcsc(n, colptr)
    np.testing.assert_array_equal(jc + 1, [int(x) for x in g["dcsc_JC"]])
    np.testing.assert_array_equal(cp + 1, [int(x) for x in g["dcsc_CP"]])
    np.testing.assert_array_equal(aux + 1, [int(x) for x in g["dcsc_AUX"]])
    assert chunk == 3
    # AUX lookup finds every column, and only the nonzero ones
    for j in range(n):
        rng = of.dcsc_lookup(j, jc, cp, aux, chunk)
        if colptr[j + 1] > colptr[j]:
            assert rng == (colptr[j], colptr[j + 1])
        else:
            assert rng is None


def test_dcsc_definition_random():
    for seed in range(20):
        A = gen.random_csc(5 + seed, 1 + 3 * seed, 0.04 + 0.01 * (seed % 7), seed)
        jc, cp, aux, chunk = of.to_dcsc(A.n, A.colptr)
        lens = np.diff(A.colptr)
        assert len(jc) == int((lens > 0).sum())
        assert len(cp) == len(jc) + 1 and cp[-1] == A.nnz
        assert aux[-1] == len(jc)
        assert np.all(np.diff(aux) >= 0)
        for j in range(A.n):
            rng = of.dcsc_lookup(j, jc, cp, aux, chunk)
            assert (rng is None) == (lens[j] == 0)
            if rng is not None:
                assert rng == (A.colptr[j], A.colptr[j + 1])


# ---------------------------------------------------------------- Fig. 8 / Section 2.4
def _fig8():
    rows = read_golden("fig8_structures.txt")
    A_rows, B_rows, C_cols, kv = {}, {}, {}, {}
    for ln in rows:
        head, _, rest = ln.partition(":")
        parts = head.split()
        if parts[0] in ("A", "B", "C") and len(parts) == 2 and ":" in ln:
            tgt = {"A": A_rows, "B": B_rows, "C": C_cols}[parts[0]]
            tgt[int(parts[1])] = [int(x) for x in rest.split()]
        else:
            kv[parts[0]] = [int(x) for x in ln.split()[1:]]
    return A_rows, B_rows, C_cols, kv


def test_fig8_flops_isect_and_pattern():
    A_rows, B_rows, C_cols, kv = _fig8()
    A = pattern_matrix(A_rows, 6, 6, by_row=True, sr=PT_I64)
    B = pattern_matrix(B_rows, 6, 6, by_row=True, sr=PT_I64, seed=3)
    # A.JC and B^T.JC printed in Section 2.4
    jcA, _, _, _ = of.to_dcsc(6, A.colptr)
    np.testing.assert_array_equal(jcA + 1, kv["A.JC"])
    tcp, _, _ = of.transpose(B.m, B.n, B.colptr, B.rowidx, B.vals)
    jcBT, _, _, _ = of.to_dcsc(6, tcp)
    np.testing.assert_array_equal(jcBT + 1, kv["BT.JC"])
    isect = np.intersect1d(jcA, jcBT)
    np.testing.assert_array_equal(isect + 1, kv["Isect"])
    # the Isect identity: sum nnz(A(:,i)) nnz(B(i,:)) = flops
    fl = oracle.flops_per_col(A, B)
    lensA = np.diff(A.colptr)
    lensBr = np.diff(tcp)
    assert int(sum(lensA[i] * lensBr[i] for i in isect)) == kv["flops"][0] == int(fl.sum())
    np.testing.assert_array_equal(fl, kv["flops_per_col"])
    for sr in SEMIRINGS:
        C = oracle.spgemm(A.with_vals(A.vals.astype(DT[sr])), B.with_vals(B.vals.astype(DT[sr])), sr)
        assert C.nnz == kv["nnzC"][0]
        for j in range(6):
            got = list(C.rowidx[C.colptr[j]:C.colptr[j + 1]] + 1)
            assert got == C_cols[j + 1]


# ---------------------------------------------------------------- Eq. 1 brute force
@pytest.mark.parametrize("sr", SEMIRINGS)
def test_bruteforce_rectangular(sr):
    rng_shapes = [(1, 1, 1), (7, 5, 3), (3, 9, 11), (12, 4, 8), (10, 10, 10), (1, 8, 6), (9, 1, 4)]
    for t, (m, k, n) in enumerate(rng_shapes):
        for dens in (0.15, 0.4, 0.9):
            A = gen.random_csc(m, k, dens, 100 * t + int(dens * 10), sr)
            B = gen.random_csc(k, n, dens, 200 * t + int(dens * 10) + 1, sr)
            if sr == PT_F64:   # mixed signs exercise cancellation paths too
                A = A.with_vals(A.vals - 0.5)
            C = oracle.spgemm(A, B, sr)
            assert_sorted_unique(C)
            ref = dense_bruteforce(A, B, sr)
            got = csc_to_dict(C)
            assert set(got) == set(ref)
            for key, v in ref.items():
                if sr == PT_F64:
                    assert abs(got[key] - v) <= 1e-14 * max(1.0, abs(v))
                else:
                    assert got[key] == v, (key, got[key], v)


def test_structural_zeros_are_kept():
    # C(0,0) = 3*2 + (-6)*1 = 0 must stay stored (structural semantics)
    A = CSC(1, 2, np.array([0, 1, 2]), np.array([0, 0], np.int32), np.array([3, -6], np.int64))
    B = CSC(2, 1, np.array([0, 2]), np.array([0, 1], np.int32), np.array([2, 1], np.int64))
    C = oracle.spgemm(A, B, PT_I64)
    assert C.nnz == 1 and C.vals[0] == 0


def test_int64_wraparound():
    big = np.int64(2 ** 62)
    A = CSC(1, 2, np.array([0, 1, 2]), np.array([0, 0], np.int32), np.array([big, big], np.int64))
    B = CSC(2, 1, np.array([0, 2]), np.array([0, 1], np.int32), np.array([2, 2], np.int64))
    C = oracle.spgemm(A, B, PT_I64)
    # 2^63 + 2^63 = 2^64 = 0 mod 2^64
    assert C.vals[0] == 0


def test_compensated_sum_exact_on_integers():
    # integer-valued doubles: every partial sum is exact, so the result is exact
    A = gen.random_csc(60, 50, 0.3, 5, PT_I64)
    B = gen.random_csc(50, 40, 0.3, 6, PT_I64)
    Ci = oracle.spgemm(A, B, PT_I64)
    Cf = oracle.spgemm(A.with_vals(A.vals.astype(np.float64)), B.with_vals(B.vals.astype(np.float64)), PT_F64)
    np.testing.assert_array_equal(Cf.vals, Ci.vals.astype(np.float64))


def test_compensated_sum_beats_naive():
    # 1 + 1e-16 * many: naive left-to-right loses every small term; Neumaier keeps them
    k = 1001
    A = CSC(1, k, np.arange(k + 1, dtype=np.int64), np.zeros(k, np.int32),
            np.array([1.0] + [1e-16] * (k - 1)))
    B = CSC(k, 1, np.array([0, k]), np.arange(k, dtype=np.int32), np.ones(k))
    C = oracle.spgemm(A, B, PT_F64)
    assert abs(C.vals[0] - (1.0 + 1e-13)) <= 1e-16


# ---------------------------------------------------------------- closed forms
def test_erdos_renyi_flops_closed_form():
    # c nonzeros in every column: flops(A*A) = c^2 n (Section 4)
    for (n, c) in ((4096, 8), (1000, 3), (257, 16)):
        A = gen.erdos_renyi(n, n, c, 0x1001 + n)
        assert np.all(np.diff(A.colptr) == c)
        fl = oracle.flops_per_col(A, A)
        assert np.all(fl == c * c)
        assert int(fl.sum()) == c * c * n
        nnz = oracle.symbolic(A, A)
        assert np.all(nnz <= np.minimum(fl, n)) and np.all(nnz >= c)


@pytest.mark.parametrize("N", [4, 8, 16])
def test_galerkin_closed_form(N):
    """R*A*P of the 7-point Laplacian with 2x2x2 aggregation is the 7-point
    operator on the coarse grid with diagonal 24 and face couplings -4."""
    A = gen.grid3d_laplacian(N)
    P = gen.aggregation_2x2x2(N)
    R = gen.transpose_host(P)
    M = N // 2
    assert A.nnz == 7 * N ** 3 - 6 * N ** 2
    AP = oracle.spgemm(A, P, PT_F64)
    assert AP.nnz == 32 * M ** 3 - 24 * M ** 2
    assert int(oracle.flops_per_col(A, P).sum()) == A.nnz
    assert int(oracle.flops_per_col(R, AP).sum()) == AP.nnz
    # AP(i, J) = 3 inside the aggregate, -1 on its outside face neighbours
    agg_of = np.empty(N ** 3, np.int64)
    for J in range(P.n):
        agg_of[P.rowidx[P.colptr[J]:P.colptr[J + 1]]] = J
    for J in range(AP.n):
        rows = AP.rowidx[AP.colptr[J]:AP.colptr[J + 1]]
        vals = AP.vals[AP.colptr[J]:AP.colptr[J + 1]]
        inside = agg_of[rows] == J
        assert np.all(vals[inside] == 3.0) and np.all(vals[~inside] == -1.0)
        assert inside.sum() == 8
    RAP = oracle.spgemm(R, AP, PT_F64)
    assert RAP.nnz == 7 * M ** 3 - 6 * M ** 2
    coarse = gen.grid3d_laplacian(M)
    np.testing.assert_array_equal(RAP.colptr, coarse.colptr)
    np.testing.assert_array_equal(RAP.rowidx, coarse.rowidx)
    np.testing.assert_array_equal(RAP.vals, 4.0 * coarse.vals)   # 6*4 = 24, -1*4 = -4


# ---------------------------------------------------------------- invariants
def _transpose(C, sr):
    tcp, tir, tv = of.transpose(C.m, C.n, C.colptr, C.rowidx, C.vals)
    return CSC(C.n, C.m, tcp, tir, tv)


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_transpose_identity(sr):
    A = gen.random_csc(40, 30, 0.1, 11, sr)
    B = gen.random_csc(30, 25, 0.15, 12, sr)
    C = oracle.spgemm(A, B, sr)
    CT = oracle.spgemm(_transpose(B, sr), _transpose(A, sr), sr)
    assert_csc_equal(_transpose(C, sr), CT, sr)


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_identity_products(sr):
    A = gen.random_csc(33, 21, 0.2, 13, sr)
    I21 = gen.identity(21, DT[sr])
    I33 = gen.identity(33, DT[sr])
    if sr == MP_F32:   # the min-plus identity has 0 on the diagonal
        I21 = I21.with_vals(np.zeros(21, np.float32))
        I33 = I33.with_vals(np.zeros(33, np.float32))
    for C in (oracle.spgemm(A, I21, sr), oracle.spgemm(I33, A, sr)):
        assert_csc_equal(C, A, sr)


@pytest.mark.parametrize("sr", [PT_I64, OR_BOOL, MP_F32])
def test_permutation_invariance(sr):
    """(P A)(B Q) = P (A B) Q exactly (Section 5.3 relabels by permutation)."""
    n = 37
    A = gen.random_csc(n, n, 0.12, 21, sr)
    B = gen.random_csc(n, n, 0.12, 22, sr)
    one = np.float32(0) if sr == MP_F32 else 1
    Pm, _ = gen.permutation_matrix(n, 5, DT[sr])
    Qm, _ = gen.permutation_matrix(n, 6, DT[sr])
    Pm = Pm.with_vals(np.full(n, one, DT[sr]))
    Qm = Qm.with_vals(np.full(n, one, DT[sr]))
    PA = oracle.spgemm(Pm, A, sr)
    BQ = oracle.spgemm(B, Qm, sr)
    lhs = oracle.spgemm(PA, BQ, sr)
    rhs = oracle.spgemm(oracle.spgemm(Pm, oracle.spgemm(A, B, sr), sr), Qm, sr)
    assert_csc_equal(lhs, rhs, sr)


@pytest.mark.parametrize("sr", [PT_I64, OR_BOOL])
def test_associativity_exact(sr):
    R = gen.random_csc(20, 45, 0.08, 31, sr)
    A = gen.random_csc(45, 45, 0.08, 32, sr)
    P = gen.random_csc(45, 17, 0.1, 33, sr)
    assert_csc_equal(oracle.spgemm(R, oracle.spgemm(A, P, sr), sr),
                     oracle.spgemm(oracle.spgemm(R, A, sr), P, sr), sr)


def test_nnz_bounds():
    A = gen.rmat(10, 8, 77)
    fl = oracle.flops_per_col(A, A)
    nz = oracle.symbolic(A, A)
    lens = np.diff(A.colptr)
    mx = np.array([lens[A.rowidx[A.colptr[j]:A.colptr[j + 1]]].max(initial=0) for j in range(A.n)])
    assert np.all(nz <= np.minimum(fl, A.m))
    assert np.all(nz >= mx)
    assert int(nz.sum()) <= int(fl.sum())


# ---------------------------------------------------------------- textbook special cases
def test_bool_bfs_step_against_adjacency_traversal():
    A = gen.rmat(11, 8, 41, OR_BOOL)
    F = gen.frontier(A.m, 16, 42, 1, 100)
    C = oracle.spgemm(A, F, OR_BOOL)
    # adjacency lists: column k of A lists the out-neighbours reached from k
    adj = [set(A.rowidx[A.colptr[k]:A.colptr[k + 1]].tolist()) for k in range(A.n)]
    for j in range(F.n):
        reach = set()
        for v in F.rowidx[F.colptr[j]:F.colptr[j + 1]].tolist():
            reach |= adj[v]
        assert sorted(reach) == C.rowidx[C.colptr[j]:C.colptr[j + 1]].tolist()
        assert np.all(C.vals[C.colptr[j]:C.colptr[j + 1]] == 1)


def test_min_plus_two_hop_relaxation():
    """(A min.+ A)(i,j) is the shortest path from j to i using exactly two edges."""
    A = gen.erdos_renyi(300, 300, 5, 51, MP_F32)
    C = oracle.spgemm(A, A, MP_F32)
    w = {}
    out_edges = {}
    for j in range(A.n):
        for p in range(A.colptr[j], A.colptr[j + 1]):
            i = int(A.rowidx[p])
            w[(i, j)] = A.vals[p]
            out_edges.setdefault(j, []).append(i)
    best = {}
    for j in range(A.n):                 # source j
        for mid in out_edges.get(j, []):  # j -> mid
            for i in out_edges.get(mid, []):  # mid -> i
                cand = np.float32(w[(mid, j)] + w[(i, mid)])
                if (i, j) not in best or cand < best[(i, j)]:
                    best[(i, j)] = cand
    assert csc_to_dict(C) == best


# ---------------------------------------------------------------- 2D blocks (Section 3.2 / 5.3)
@pytest.mark.parametrize("g", [1, 3, 4, 7])
def test_partition_reassembles_and_block_products_sum(g):
    sr = PT_I64
    A = gen.random_csc(29, 23, 0.12, 61, sr)
    B = gen.random_csc(23, 26, 0.12, 62, sr)
    blocksA = of.partition(A.m, A.n, A.colptr, A.rowidx, A.vals, g)
    blocksB = of.partition(B.m, B.n, B.colptr, B.rowidx, B.vals, g)
    # reassembly equals the input
    back = {}
    for (I, J), (r0, r1, c0, c1, cp, ir, nv) in blocksA.items():
        for jj in range(c1 - c0):
            for p in range(cp[jj], cp[jj + 1]):
                back[(int(ir[p]) + r0, jj + c0)] = nv[p]
    assert back == csc_to_dict(A)
    # C_IJ = sum_K A_IK B_KJ equals the flat product's block (Sparse SUMMA, Section 3.5)
    flat = csc_to_dict(oracle.spgemm(A, B, sr))
    acc = {}
    for I in range(g):
        for J in range(g):
            for K in range(g):
                r0, r1, k0, k1, cpa, ira, nva = blocksA[(I, K)]
                _, _, c0, c1, cpb, irb, nvb = blocksB[(K, J)]
                if r1 <= r0 or c1 <= c0 or k1 <= k0:
                    continue
                P = oracle.spgemm(CSC(r1 - r0, k1 - k0, cpa, ira, nva), CSC(k1 - k0, c1 - c0, cpb, irb, nvb), sr)
                for (i, j), v in csc_to_dict(P).items():
                    key = (i + r0, j + c0)
                    acc[key] = acc.get(key, 0) + int(v)
    assert acc == {k: int(v) for k, v in flat.items()}


def test_spgemm_columns_subset_matches_full():
    A = gen.rmat(9, 8, 71)
    C = oracle.spgemm(A, A, PT_F64)
    cols = np.array([0, 5, 17, 511, 300])
    S = oracle.spgemm_columns(A, A, PT_F64, cols)
    for t, j in enumerate(cols):
        np.testing.assert_array_equal(S.rowidx[S.colptr[t]:S.colptr[t + 1]], C.rowidx[C.colptr[j]:C.colptr[j + 1]])
        np.testing.assert_array_equal(S.vals[S.colptr[t]:S.colptr[t + 1]], C.vals[C.colptr[j]:C.colptr[j + 1]])


def test_threads_do_not_change_result():
    A = gen.rmat(10, 8, 81)
    C1 = oracle.spgemm(A, A, PT_F64, nthreads=1)
    C4 = oracle.spgemm(A, A, PT_F64, nthreads=4)
    np.testing.assert_array_equal(C1.rowidx, C4.rowidx)
    np.testing.assert_array_equal(C1.vals, C4.vals)


def test_permute_definition_and_pcpt_identity():
    """permute moves A(i,j) to (p[i], q[j]) (checked on dense arrays), the inverse
    permutation undoes it, and (PAP^T)(PAP^T) = P(AA)P^T exactly (Section 5.3.3)."""
    A = gen.random_csc(40, 40, 0.12, 0x51, PT_I64)
    p = np.random.default_rng(5).permutation(40)
    q = np.random.default_rng(6).permutation(40)
    cp, ir, v = of.permute(A.m, A.n, A.colptr, A.rowidx, A.vals, p, q)
    dense_a = np.zeros((40, 40), np.int64)
    for j in range(40):
        dense_a[A.rowidx[A.colptr[j]:A.colptr[j + 1]], j] = A.vals[A.colptr[j]:A.colptr[j + 1]]
    dense_b = np.zeros((40, 40), np.int64)
    for j in range(40):
        seg = slice(cp[j], cp[j + 1])
        assert np.all(np.diff(ir[seg]) > 0)
        dense_b[ir[seg], j] = v[seg]
    assert np.array_equal(dense_b[np.ix_(p, q)], dense_a)
    back = of.permute(40, 40, cp, ir, v, np.argsort(p), np.argsort(q))
    assert np.array_equal(back[0], A.colptr) and np.array_equal(back[1], A.rowidx) and np.array_equal(back[2], A.vals)
    B = gen.rmat(9, 8, 0x52, PT_I64)
    p = np.random.default_rng(7).permutation(B.n)
    Bp = CSC(B.m, B.n, *of.permute(B.m, B.n, B.colptr, B.rowidx, B.vals, p, p))
    C = oracle.spgemm(B, B, PT_I64)
    Cp = oracle.spgemm(Bp, Bp, PT_I64)
    ref = of.permute(C.m, C.n, C.colptr, C.rowidx, C.vals, p, p)
    assert np.array_equal(Cp.colptr, ref[0]) and np.array_equal(Cp.rowidx, ref[1]) and np.array_equal(Cp.vals, ref[2])


# ---------------------------------------------------------------- second oracle: H_GEMM (Section 2.4)
def test_hgemm_fig8_isect_flops_and_pattern():
    """The heap-merged outer products on the Fig. 8 operands: the printed Isect,
    the flops identity (19) and the pattern of C by column."""
    from oracle import hgemm as oh
    A_rows, B_rows, C_cols, kv = _fig8()
    A = pattern_matrix(A_rows, 6, 6, by_row=True, sr=PT_I64)
    B = pattern_matrix(B_rows, 6, 6, by_row=True, sr=PT_I64, seed=3)
    tcp = of.transpose(B.m, B.n, B.colptr, B.rowidx, B.vals)[0]
    assert [i + 1 for i in oh.isect(A.colptr, tcp)] == list(kv["Isect"])
    assert oh.flops(A, B) == kv["flops"][0]
    cp, ir, v = oh.hgemm(A, B, PT_I64)
    for j in range(6):
        assert list(ir[cp[j]:cp[j + 1]] + 1) == C_cols[j + 1]


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_hgemm_equals_gustavson(sr):
    """Two independent formulations of C = A*B (heap merge of outer products vs
    column-wise SPA) agree: structure and exact semirings bit for bit, FP64 within
    the tolerance."""
    from oracle import hgemm as oh
    cases = [(gen.random_csc(23, 17, 0.2, 0x61, sr), gen.random_csc(17, 29, 0.15, 0x62, sr)),
             (gen.rmat(7, 6, 0x63, sr), gen.rmat(7, 6, 0x64, sr)),
             (gen.random_csc(40, 60, 0.02, 0x65, sr), gen.random_csc(60, 30, 0.03, 0x66, sr))]   # hypersparse
    for A, B in cases:
        R = oracle.spgemm(A, B, sr)
        cp, ir, v = oh.hgemm(A, B, sr)
        np.testing.assert_array_equal(cp, R.colptr)
        np.testing.assert_array_equal(ir, R.rowidx)
        if sr == PT_F64:
            assert np.all(np.abs(v - R.vals) <= FP64_RTOL * np.abs(R.vals))
        else:
            np.testing.assert_array_equal(v, R.vals)
