"""Parity of the flat CUDA product (plan -> symbolic -> numeric) with the CPU oracle."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_matches, check_product, gpu_product, sp
from helpers import MP_F32, OR_BOOL, PT_F64, PT_I64
from paper_1006_2183_gb300 import gen
from paper_1006_2183_gb300.gen import CSC

pytestmark = pytest.mark.gpu
SEMIRINGS = [PT_F64, MP_F32, OR_BOOL, PT_I64]


@pytest.fixture(scope="module")
def ctx():
    s = sp()
    return s.Context()


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_er_4096_eight_per_column(ctx, sr):
    """C = A*A, A 4096 x 4096 ER with exactly 8 per column (full comparison)."""
    A = gen.erdos_renyi(4096, 4096, 8, 0x1001, sr)
    C = check_product(ctx, A, A, sr)
    fl = oracle.flops_per_col(A, A)
    assert int(fl.sum()) == 8 * 8 * 4096


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_rectangular_random(ctx, sr):
    for t, (m, k, n, dens) in enumerate([(37, 29, 41, 0.1), (300, 200, 150, 0.03), (1, 50, 70, 0.3),
                                         (90, 1, 33, 0.5), (513, 257, 129, 0.02), (2000, 3000, 100, 0.01)]):
        A = gen.random_csc(m, k, dens, 10 + t, sr)
        B = gen.random_csc(k, n, dens, 20 + t, sr)
        if sr == PT_F64:
            A = A.with_vals(A.vals - 0.5)   # cancellation on the way
        check_product(ctx, A, B, sr, what=f"shape {(m, k, n)}")


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_rmat_all_tiers(ctx, sr):
    """R-MAT scale 13: columns land in every tier (warp, CTA hash, dense chunks)."""
    A = gen.rmat(13, 8, 0x1302, sr)
    C = check_product(ctx, A, A, sr)
    s = sp()
    dA = s.Matrix.from_host(ctx, A, sr)
    plan = s.spgemm_plan(ctx, dA, dA, sr)
    st = plan.stats()
    assert st["tiers"][1] > 0 and st["tiers"][2] > 0 and st["tiers"][3] > 0, st
    assert st["flops"] == int(oracle.flops_per_col(A, A).sum())


def test_bool_with_stored_false_values(ctx):
    """Boolean operands that store false entries (0 bytes) and other true bytes (2):
    stored false entries still make structural entries of C, whose values are
    the OR of the ANDs; long columns then evaluate every product instead of
    taking every output as true."""
    A = gen.rmat(13, 8, 0x1303, OR_BOOL)
    v = np.where(np.arange(A.nnz) % 3 == 0, 0, np.where(np.arange(A.nnz) % 3 == 1, 1, 2)).astype(np.uint8)
    A = A.with_vals(v)
    C = check_product(ctx, A, A, OR_BOOL)
    s = sp()
    dA = s.Matrix.from_host(ctx, A, OR_BOOL)
    assert s.spgemm_plan(ctx, dA, dA, OR_BOOL).stats()["tiers"][3] > 0   # long columns present
    assert (C.vals == 0).any() and (C.vals == 1).any()


@pytest.mark.parametrize("sr", [PT_F64, PT_I64])
def test_tier_choice_does_not_change_result(ctx, sr):
    A = gen.rmat(12, 8, 0x1202, sr)
    s = sp()
    ref = oracle.spgemm(A, A, sr)
    for kw in ({"warp_max_flops": 0, "block_max_flops": 0},      # everything dense
               {"warp_max_flops": 512, "block_max_flops": 4096},
               {"warp_max_flops": 0, "block_max_flops": 4096},    # CTA tables only
               {"dense_part_flops": 1024}):                       # many dense parts
        C = gpu_product(ctx, A, A, sr, s.default_opts(**kw))
        assert_matches(C, ref, sr, what=str(kw))


@pytest.mark.parametrize("sr", [PT_F64, MP_F32])
def test_slab_rows_do_not_change_result(ctx, sr):
    """Long columns cut into row slabs of 4096 .. 65536 rows (up to the 16-slab limit,
    which raises the slab size for 2^16 rows / 4096) give the same result; 2^16 rows
    keep the long columns in the range tier."""
    A = gen.rmat(16, 8, 0x1602, sr)
    s = sp()
    ref = oracle.spgemm(A, A, sr)
    for rows in (4096, 8192, 1000, 65536, 0):
        C = gpu_product(ctx, A, A, sr, s.default_opts(range_slab_rows=rows, dense_part_flops=1024))
        assert_matches(C, ref, sr, what=f"slab rows {rows}")


@pytest.mark.parametrize("sr", [PT_F64, OR_BOOL])
def test_tall_long_columns_cut_into_slabs(ctx, sr):
    """3,000,017 rows: long columns need at least 6 row slabs of 2^19 rows (ragged last
    slab); columns of 1, 2 and 64 B entries cover the hash and range tiers."""
    s = sp()
    m, k = 3_000_017, 64
    rng = np.random.default_rng(3)
    cp = np.zeros(k + 1, np.int64)
    ir = []
    for c in range(k):
        u = np.unique(rng.integers(0, m, 150 if c % 2 else 90)).astype(np.int32)
        if c == 5:
            u = np.unique(np.concatenate([u, np.array([0, m - 1], np.int32)]))   # first and last row
        ir.append(u)
        cp[c + 1] = cp[c] + len(u)
    irs = np.concatenate(ir)
    vals = rng.random(len(irs)) if sr == PT_F64 else np.ones(len(irs), np.uint8)
    A = CSC(m, k, cp, irs, vals)
    B = CSC(k, 4, np.array([0, 1, 3, 67, 131], np.int64),
            np.concatenate([[5], [2, 9], np.arange(64), np.arange(64)]).astype(np.int32),
            rng.random(131) if sr == PT_F64 else np.ones(131, np.uint8))
    C = s.spgemm_multiply(ctx, s.Matrix.from_host(ctx, A, sr), s.Matrix.from_host(ctx, B, sr), sr).to_host()
    assert_matches(C, oracle.spgemm(A, B, sr), sr, what="tall slabs")


@pytest.mark.parametrize("sr", SEMIRINGS)
def test_dense_column_tier_boundaries(ctx, sr):
    """Long columns on both sides of the dense-column limit (16384 rows for 8-byte
    accumulators, 32768 for 4-byte ones): the dense row array below, the range tier
    above, the same result as the oracle either way."""
    s = sp()
    for m in (16384, 16385, 32768, 32769):
        A = gen.erdos_renyi(m, 96, 120, 0xD0 + m % 7, sr)
        B = gen.erdos_renyi(96, 24, 60, 0xD1 + m % 5, sr)   # 60 x 120 = 7200 products per column
        check_product(ctx, A, B, sr, what=f"m = {m}")


def _tall_a(m, k=64, seed=17):
    rng = np.random.default_rng(seed)
    rows = rng.choice(m, (k, 100), replace=True)
    cp = np.zeros(k + 1, np.int64)
    ir = []
    for c in range(k):
        u = np.unique(rows[c]).astype(np.int32)
        ir.append(u)
        cp[c + 1] = cp[c] + len(u)
    return CSC(m, k, cp, np.concatenate(ir), np.ones(int(cp[-1])))


def test_long_column_of_many_slabs_matches_oracle(ctx):
    """A long column of 17 * 2^20 rows needs 35 row slabs of at most 2^19 rows (the
    slab count stays under its limit of 64); it matches the oracle, as do short
    columns of the same tall A."""
    s = sp()
    A = _tall_a(17 * (1 << 20))
    k = A.n
    dA = s.Matrix.from_host(ctx, A, PT_F64)
    long_b = CSC(k, 1, np.array([0, k], np.int64), np.arange(k, dtype=np.int32), np.ones(k))   # ~6400 flops
    C = s.spgemm_multiply(ctx, dA, s.Matrix.from_host(ctx, long_b, PT_F64), PT_F64).to_host()
    assert_matches(C, oracle.spgemm(A, long_b, PT_F64), PT_F64, what="one long column over 35 slabs")
    short_b = CSC(k, 2, np.array([0, 2, 3], np.int64), np.array([1, 5, 9], np.int32), np.ones(3))
    C = s.spgemm_multiply(ctx, dA, s.Matrix.from_host(ctx, short_b, PT_F64), PT_F64).to_host()
    assert_matches(C, oracle.spgemm(A, short_b, PT_F64), PT_F64, what="short columns of a tall A")


def test_long_column_over_slab_limit_is_unsupported(ctx):
    """A long column of more than 64 * (2^20 - 32) rows is refused, not cut into slabs
    wider than the shared-memory bitmap."""
    s = sp()
    A = _tall_a(65 * (1 << 20))
    k = A.n
    dA = s.Matrix.from_host(ctx, A, PT_F64)
    long_b = CSC(k, 1, np.array([0, k], np.int64), np.arange(k, dtype=np.int32), np.ones(k))
    with pytest.raises(s.SpGEMMError) as ei:
        s.spgemm_multiply(ctx, dA, s.Matrix.from_host(ctx, long_b, PT_F64), PT_F64)
    assert ei.value.status == 8, ei.value   # SPGEMM_ERR_UNSUPPORTED


def test_dense_rows_multiple_chunks_and_ragged_tail(ctx):
    # m not a multiple of the dense chunk (8192 rows for FP64): several chunks and a short tail
    m = 3 * 8192 + 77
    A = gen.erdos_renyi(m, 400, 60, 5)
    B = gen.erdos_renyi(400, 50, 200, 6)
    check_product(ctx, A, B, PT_F64, what="dense with tail")


def test_edge_cases(ctx):
    s = sp()
    sr = PT_F64
    # empty matrices
    Z = CSC(5, 7, np.zeros(8, np.int64), np.zeros(0, np.int32), np.zeros(0))
    Y = CSC(7, 3, np.zeros(4, np.int64), np.zeros(0, np.int32), np.zeros(0))
    C = gpu_product(ctx, Z, Y, sr)
    assert C.nnz == 0 and list(C.colptr) == [0, 0, 0, 0]
    # 1 x 1
    one = CSC(1, 1, np.array([0, 1]), np.array([0], np.int32), np.array([3.0]))
    C = gpu_product(ctx, one, one, sr)
    assert C.nnz == 1 and C.vals[0] == 9.0
    # one dense column times a row of ones
    m = 5000
    D = CSC(m, 1, np.array([0, m]), np.arange(m, dtype=np.int32), np.linspace(0, 1, m))
    Rw = CSC(1, 40, np.arange(41, dtype=np.int64), np.zeros(40, np.int32), np.arange(1.0, 41.0))
    check_product(ctx, D, Rw, sr, what="outer product")
    # columns exactly at the warp/CTA thresholds: flops 512 and 4096
    for f in (32, 512, 513, 4096, 4097):
        A = gen.erdos_renyi(20000, 64, 64, 7)
        cnt = f // 64
        B = gen.erdos_renyi(64, 3, max(cnt, 1), 8 + f)
        check_product(ctx, A, B, sr, what=f"flops ~{f}")


@pytest.mark.parametrize("sr", [PT_F64, OR_BOOL])
def test_csr_and_dcsc_operands(ctx, sr):
    s = sp()
    A = gen.rmat(10, 8, 31, sr)
    B = gen.random_csc(1024, 300, 0.004, 32, sr)
    R = oracle.spgemm(A, B, sr)
    dA = s.Matrix.from_host(ctx, A, sr)
    dB = s.Matrix.from_host(ctx, B, sr)
    # A given as CSR (its transpose's CSC arrays)
    from oracle import formats as of
    tcp, tir, tv = of.transpose(A.m, A.n, A.colptr, A.rowidx, A.vals)
    import torch
    dev = ctx.device
    Acsr = s.Matrix.csr(ctx, A.m, A.n, torch.from_numpy(tcp).to(dev), torch.from_numpy(tir).to(dev),
                        torch.from_numpy(np.ascontiguousarray(tv)).to(dev), sr)
    assert_matches(s.spgemm_multiply(ctx, Acsr, dB, sr).to_host(), R, sr, what="A csr")
    # B as DCSC (hypersparse: most of its columns are empty), A as DCSC with AUX
    Bd = s.spgemm_mat_to_dcsc(ctx, dB, True)
    assert_matches(s.spgemm_multiply(ctx, dA, Bd, sr).to_host(), R, sr, what="B dcsc")
    Ad = s.spgemm_mat_to_dcsc(ctx, dA, True)
    assert_matches(s.spgemm_multiply(ctx, Ad, Bd, sr).to_host(), R, sr, what="A,B dcsc")


def test_transpose_and_dcsc_against_oracle(ctx):
    from oracle import formats as of
    s = sp()
    for seed, (m, n, d) in enumerate([(300, 200, 0.02), (4000, 4096, 0.0005), (1, 9, 0.5), (9, 9, 0.05)]):
        A = gen.random_csc(m, n, d, 40 + seed)
        dA = s.Matrix.from_host(ctx, A, PT_F64)
        T = s.spgemm_mat_transpose(ctx, dA).to_host()
        tcp, tir, tv = of.transpose(A.m, A.n, A.colptr, A.rowidx, A.vals)
        np.testing.assert_array_equal(T.colptr, tcp)
        np.testing.assert_array_equal(T.rowidx, tir)
        np.testing.assert_array_equal(T.vals, tv)
        D = s.spgemm_mat_to_dcsc(ctx, dA, True)
        nzc, jc, aux, chunk = D.export_dcsc()
        ojc, ocp, oaux, ochunk = of.to_dcsc(A.n, A.colptr)
        assert nzc == len(ojc) and chunk == ochunk
        np.testing.assert_array_equal(jc.cpu().numpy(), ojc)
        np.testing.assert_array_equal(aux.cpu().numpy(), oaux)
        np.testing.assert_array_equal(D.export()[3].cpu().numpy(), ocp)


def test_nine_by_nine_dcsc_example(ctx):
    """The DCSC of the 9x9 example of Section 2.3 (JC, CP, AUX) from the device converter."""
    s = sp()
    cp, ir = gen.csc_from_coo(9, 9, np.array([5, 7, 3, 1]), np.array([0, 0, 6, 7]))
    A = CSC(9, 9, cp, ir, np.array([0.1, 0.2, 0.3, 0.4]))
    D = s.spgemm_mat_to_dcsc(ctx, s.Matrix.from_host(ctx, A, PT_F64), True)
    nzc, jc, aux, chunk = D.export_dcsc()
    assert list(jc.cpu().numpy() + 1) == [1, 7, 8]
    assert list(D.export()[3].cpu().numpy() + 1) == [1, 3, 4, 5]
    assert list(aux.cpu().numpy() + 1) == [1, 2, 2, 4]


def test_errors_are_reported(ctx):
    s = sp()
    import torch
    dev = ctx.device
    A = gen.random_csc(10, 8, 0.3, 1)
    B = gen.random_csc(9, 4, 0.3, 2)
    dA, dB = s.Matrix.from_host(ctx, A, PT_F64), s.Matrix.from_host(ctx, B, PT_F64)
    with pytest.raises(s.SpGEMMError) as e:
        s.spgemm_multiply(ctx, dA, dB, PT_F64)
    assert e.value.status == 2   # DIM_MISMATCH
    with pytest.raises(s.SpGEMMError):
        s.spgemm_multiply(ctx, dA, dA.__class__.from_host(ctx, gen.random_csc(8, 4, 0.3, 3), PT_I64), PT_F64)
    # unsorted rows inside a column -> BAD_FORMAT from the validator
    bad = s.Matrix.csc(ctx, 4, 1, torch.tensor([0, 2], dtype=torch.int64, device=dev),
                       torch.tensor([3, 1], dtype=torch.int32, device=dev), torch.ones(2, dtype=torch.float64, device=dev),
                       PT_F64)
    with pytest.raises(s.SpGEMMError) as e:
        bad.validate()
    assert e.value.status == 3
    oob = s.Matrix.csc(ctx, 4, 1, torch.tensor([0, 1], dtype=torch.int64, device=dev),
                       torch.tensor([9], dtype=torch.int32, device=dev), torch.ones(1, dtype=torch.float64, device=dev),
                       PT_F64)
    with pytest.raises(s.SpGEMMError):
        oob.validate()
    dA.validate()


def test_symbolic_matches_oracle_counts(ctx):
    s = sp()
    A = gen.rmat(12, 8, 0x77)
    dA = s.Matrix.from_host(ctx, A, PT_F64)
    plan = s.spgemm_plan(ctx, dA, dA, PT_F64)
    nnz = s.spgemm_symbolic(plan)
    ref = oracle.symbolic(A, A)
    assert nnz == int(ref.sum())
    C = s.spgemm_numeric(plan).to_host()
    np.testing.assert_array_equal(np.diff(C.colptr), ref)


@pytest.mark.parametrize("sr", [PT_F64, MP_F32])
def test_rmat_scale18_sampled(ctx, sr):
    """The benchmark workload (R-MAT scale 18, edge factor 8): sampled columns vs the oracle,
    plus whole-matrix properties (nnz <= min(flops, m), rows sorted, nnz = oracle symbolic)."""
    A = gen.rmat(18, 8, 0x1802, sr)
    s = sp()
    dA = s.Matrix.from_host(ctx, A, sr)
    C = s.spgemm_multiply(ctx, dA, dA, sr).to_host()
    nz = oracle.symbolic(A, A)
    np.testing.assert_array_equal(np.diff(C.colptr), nz)
    lens = np.diff(A.colptr)
    rng = np.random.default_rng(1)
    heavy = np.argsort(lens)[-20:]
    cols = np.unique(np.concatenate([heavy, rng.choice(A.n, 300, replace=False), [0, A.n - 1]]))
    R = oracle.spgemm_columns(A, A, sr, cols)
    for t, j in enumerate(cols):
        got_r = C.rowidx[C.colptr[j]:C.colptr[j + 1]]
        np.testing.assert_array_equal(got_r, R.rowidx[R.colptr[t]:R.colptr[t + 1]])
        got_v = C.vals[C.colptr[j]:C.colptr[j + 1]]
        ref_v = R.vals[R.colptr[t]:R.colptr[t + 1]]
        if sr == PT_F64:
            assert np.all(np.abs(got_v - ref_v) <= 1e-13 * np.abs(ref_v)), j
        else:
            np.testing.assert_array_equal(got_v, ref_v)
    col_of = np.repeat(np.arange(C.n), np.diff(C.colptr))
    same = col_of[1:] == col_of[:-1]
    assert np.all(np.diff(C.rowidx.astype(np.int64))[same] > 0)


def test_repeatable_exact_semirings(ctx):
    A = gen.rmat(12, 8, 0x99, PT_I64)
    C1 = gpu_product(ctx, A, A, PT_I64)
    C2 = gpu_product(ctx, A, A, PT_I64)
    np.testing.assert_array_equal(C1.vals, C2.vals)


def test_malformed_operands_are_refused_before_any_product_kernel(ctx):
    """Section 8(b) preconditions: a non-monotone colptr, rows out of order and a
    row past m are reported as SPGEMM_ERR_BAD_FORMAT by the input check of the
    product call (the default), so no product kernel reads the arrays; a valid
    operand then works on the same context, and check_inputs = 0 skips the check."""
    s = sp()
    A = gen.random_csc(50, 40, 0.1, 77)
    good = s.Matrix.from_host(ctx, A, PT_F64)
    cp = A.colptr.copy()
    cp[10], cp[11] = cp[11], cp[10] - 1                       # colptr decreases
    rows = A.rowidx.copy()
    j = int(np.argmax(np.diff(A.colptr) >= 2))
    s0 = A.colptr[j]
    rows[s0], rows[s0 + 1] = rows[s0 + 1], rows[s0]           # two rows of one column swapped
    past = A.rowidx.copy()
    past[-1] = A.m + 3                                         # a row past m
    for name, M in (("non-monotone colptr", CSC(A.m, A.n, cp, A.rowidx, A.vals)),
                    ("unsorted rows", CSC(A.m, A.n, A.colptr, rows, A.vals)),
                    ("row past m", CSC(A.m, A.n, A.colptr, past, A.vals))):
        bad = s.Matrix.from_host(ctx, M, PT_F64)
        At = s.Matrix.from_host(ctx, gen.transpose_host(A), PT_F64)   # 40 x 50: At * bad is defined
        with pytest.raises(s.SpGEMMError) as ei:
            s.spgemm_multiply(ctx, At, bad, PT_F64)
        assert ei.value.status == 3, (name, ei.value)
        with pytest.raises(s.SpGEMMError) as ei:
            s.spgemm_summa_blocked(ctx, At, bad, 4, PT_F64)
        assert ei.value.status == 3, (name, ei.value)
        with pytest.raises(s.SpGEMMError) as ei:
            s.spgemm_batch(ctx, [At], [bad], PT_F64)
        assert ei.value.status == 3, (name, ei.value)
    # the context still works, and a checked handle is not checked again
    At = s.Matrix.from_host(ctx, gen.transpose_host(A), PT_F64)
    C = s.spgemm_multiply(ctx, At, good, PT_F64).to_host()
    assert_matches(C, oracle.spgemm(gen.transpose_host(A), A, PT_F64), PT_F64, what="after refused operands")
    C = s.spgemm_multiply(ctx, At, good, PT_F64, s.default_opts(check_inputs=0)).to_host()
    assert_matches(C, oracle.spgemm(gen.transpose_host(A), A, PT_F64), PT_F64, what="check_inputs = 0")


def _quad_edge_case(seed):
    """A of 40000 rows (slab tier) whose last column holds the array's last entries,
    nnz = 3 mod 4, and one long B column over every column of A (the quad walk's
    partial last quad); plus a short B column."""
    rng = np.random.default_rng(seed)
    m, k = 40000, 300
    cols = [np.sort(rng.choice(m, int(rng.integers(20, 80)), replace=False)).astype(np.int32) for _ in range(k)]
    while sum(len(c) for c in cols) % 4 != 3:
        cols[-1] = np.sort(np.unique(np.append(cols[-1], rng.integers(0, m)))).astype(np.int32)
    cp = np.zeros(k + 1, np.int64)
    np.cumsum([len(c) for c in cols], out=cp[1:])
    A = CSC(m, k, cp, np.concatenate(cols), rng.uniform(0, 1, int(cp[-1])))
    B = CSC(k, 2, np.array([0, k, k + 2], np.int64), np.concatenate([np.arange(k), [k - 2, k - 1]]).astype(np.int32),
            rng.uniform(0, 1, k + 2))
    return A, B


@pytest.mark.parametrize("sr", [PT_F64, OR_BOOL, PT_I64])
def test_slab_quads_partial_last_quad(ctx, sr):
    A, B = _quad_edge_case(91)
    A = A.with_vals(gen.values_for(sr, 5, A.nnz)) if sr != PT_F64 else A
    B = B.with_vals(gen.values_for(sr, 6, B.nnz)) if sr != PT_F64 else B
    s = sp()
    dA = s.Matrix.from_host(ctx, A, sr)
    assert s.spgemm_plan(ctx, dA, s.Matrix.from_host(ctx, B, sr), sr).stats()["tiers"][3] == 1
    check_product(ctx, A, B, sr, what="partial last quad")


def test_slab_misaligned_arrays_take_the_scalar_walk(ctx):
    """Row and value arrays that start 4 and 8 bytes past a 16-byte boundary (views
    into larger tensors): the long column is walked one product per lane."""
    import torch
    A, B = _quad_edge_case(92)
    s = sp()
    dev = ctx.device
    ir = torch.zeros(A.nnz + 1, dtype=torch.int32, device=dev)
    ir[1:] = torch.from_numpy(A.rowidx).to(dev)
    v = torch.zeros(A.nnz + 1, dtype=torch.float64, device=dev)
    v[1:] = torch.from_numpy(A.vals).to(dev)
    cp = torch.from_numpy(A.colptr).to(dev)
    assert ir[1:].data_ptr() % 16 == 4 and v[1:].data_ptr() % 16 == 8
    dA = s.Matrix.csc(ctx, A.m, A.n, cp, ir[1:], v[1:], PT_F64)
    C = s.spgemm_multiply(ctx, dA, s.Matrix.from_host(ctx, B, PT_F64), PT_F64).to_host()
    assert_matches(C, oracle.spgemm(A, B, PT_F64), PT_F64, what="misaligned A")
