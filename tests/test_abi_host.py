"""Host-side argument checks of the C ABI, on the CPU: every call below returns its
status before any device work, so no GPU is needed."""
import ctypes

import pytest

from helpers import GOLDEN  # noqa: F401  (sets up sys.path through conftest)

OK, INVALID_ARG, INDEX_OVERFLOW = 0, 1, 5
P = ctypes.c_void_p
PP = ctypes.POINTER(ctypes.c_void_p)
I64 = ctypes.c_int64


@pytest.fixture(scope="module")
def lib():
    from paper_1006_2183_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.spgemm_status_string.restype = ctypes.c_char_p
    lib.spgemm_status_string.argtypes = [ctypes.c_int]
    lib.spgemm_last_error.restype = ctypes.c_char_p
    lib.spgemm_last_error.argtypes = [P]
    lib.spgemm_ctx_create.argtypes = [PP, P, P, P, P]
    lib.spgemm_ctx_destroy.argtypes = [P]
    lib.spgemm_mat_csc.argtypes = [P, PP, I64, I64, I64, P, P, P, ctypes.c_int]
    lib.spgemm_mat_destroy.argtypes = [P]
    lib.spgemm_summa_blocked.argtypes = [P, P, P, ctypes.c_int, ctypes.c_int, P, PP]
    lib.spgemm_summa_pipelined.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_int, P, PP]
    lib.spgemm_multiply.argtypes = [P, P, P, ctypes.c_int, P, PP]
    return lib


@pytest.fixture(scope="module")
def ctx(lib):
    h = P()
    assert lib.spgemm_ctx_create(ctypes.byref(h), None, None, None, None) == OK
    yield h
    lib.spgemm_ctx_destroy(h)


def test_status_strings(lib):
    names = [lib.spgemm_status_string(s).decode() for s in range(10)]
    assert names[0] == "ok" and all(names) and len(set(names)) == 10


def test_context_creation_checks(lib):
    h = P()
    assert lib.spgemm_ctx_create(None, None, None, None, None) == INVALID_ARG
    # an allocator without its free function (or the reverse) is refused
    assert lib.spgemm_ctx_create(ctypes.byref(h), None, P(1), None, None) == INVALID_ARG
    assert lib.spgemm_ctx_create(ctypes.byref(h), None, None, P(1), None) == INVALID_ARG


def test_matrix_handle_checks(lib, ctx):
    h = P()
    fake = P(256)   # never dereferenced: handles borrow arrays unchecked
    assert lib.spgemm_mat_csc(ctx, ctypes.byref(h), -1, 4, 0, fake, fake, fake, 0) == INVALID_ARG
    assert lib.spgemm_mat_csc(ctx, ctypes.byref(h), 1 << 31, 4, 0, fake, fake, fake, 0) == INDEX_OVERFLOW
    assert lib.spgemm_mat_csc(ctx, ctypes.byref(h), 4, 4, 3, None, fake, fake, 0) == INVALID_ARG
    assert lib.spgemm_mat_csc(ctx, ctypes.byref(h), 4, 4, 3, fake, None, fake, 0) == INVALID_ARG
    assert lib.spgemm_mat_csc(ctx, ctypes.byref(h), 4, 4, 3, fake, fake, fake, 9) == INVALID_ARG   # semiring
    assert lib.spgemm_last_error(ctx)
    assert lib.spgemm_mat_csc(ctx, ctypes.byref(h), 4, 4, 3, fake, fake, fake, 3) == OK
    assert lib.spgemm_mat_destroy(h) == OK


def test_product_entry_points_check_their_handles(lib, ctx):
    out = P()
    assert lib.spgemm_multiply(None, None, None, 0, None, ctypes.byref(out)) == INVALID_ARG
    assert lib.spgemm_summa_blocked(None, None, None, 4, 0, None, ctypes.byref(out)) == INVALID_ARG
    assert lib.spgemm_summa_pipelined(ctx, None, None, None, 4, 0, None, ctypes.byref(out)) == INVALID_ARG
    # the merge context must be a second context
    h = P()
    fake = P(256)
    assert lib.spgemm_mat_csc(ctx, ctypes.byref(h), 4, 4, 3, fake, fake, fake, 0) == OK
    assert lib.spgemm_summa_pipelined(ctx, ctx, h, h, 4, 0, None, ctypes.byref(out)) == INVALID_ARG
    assert b"second context" in lib.spgemm_last_error(ctx)
    lib.spgemm_mat_destroy(h)


def test_default_options():
    from paper_1006_2183_gb300 import spgemm as sp
    o = sp.default_opts()
    assert (o.warp_max_flops, o.block_max_flops, o.dense_part_flops) == (512, -1, 65536)
    assert (o.use_predictor, o.summa_fused, o.summa_merge_every, o.block_kernel, o.range_slab_rows) == (0, 0, 0, 0, 0)


def test_colptr_noalloc_rejects_null_arrays_before_any_cuda_call(lib):
    """A null row-index array is refused by the argument checks, so no kernel can
    read through it; those checks run before the first CUDA call (no GPU here)."""
    lib.spgemm_colptr_noalloc.argtypes = [P, I64, I64, I64, P, P, P, P, P]
    fake = P(256)
    args = [None, 8, 8, 8, fake, fake, fake, fake, fake]
    assert lib.spgemm_colptr_noalloc(*args[:5], None, *args[6:]) == INVALID_ARG      # Arowidx
    assert lib.spgemm_colptr_noalloc(*args[:7], None, args[8]) == INVALID_ARG        # Browidx
    assert lib.spgemm_colptr_noalloc(*args[:4], None, *args[5:]) == INVALID_ARG      # Acolptr
    assert lib.spgemm_colptr_noalloc(*args[:8], None) == INVALID_ARG                 # Ccolptr
    assert lib.spgemm_colptr_noalloc(None, -1, 8, 8, fake, fake, fake, fake, fake) == INVALID_ARG
