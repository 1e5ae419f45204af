"""The no-allocation entry point (spgemm_colptr_noalloc).

Callers that cannot allocate device memory where they need C's structure -- a
fixed, pre-planned memory budget, a latency-critical path that must not make
allocation calls, or a plugin whose host program owns all device memory -- get
C's column pointers from spgemm_colptr_noalloc, which touches only the
caller's arrays and one small static scratch array.  These tests check its
output against the oracle's symbolic pass and against the regular symbolic pass
(spgemm_multiply's column pointers), exactly, on two calls in a row (the second
call reuses the scratch array the first one left behind), on the tall and wide
shapes that take its other code paths, and that sizes beyond its limits are
refused.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import oracle

from gpu_util import sp
from helpers import PT_F64
from paper_1006_2183_gb300 import gen

pytestmark = pytest.mark.gpu


def _dev(a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()


def test_colptr_noalloc_matches_oracle_and_regular_symbolic_on_two_calls():
    s = sp()
    stream = torch.cuda.Stream()
    ctx = s.Context(stream=stream)
    cases = [(gen.rmat(12, 8, 0x2201), None),                                           # square, skewed
             (gen.erdos_renyi(5000, 300, 7, 0x2202), gen.erdos_renyi(300, 9000, 3, 0x2203))]  # rectangular, n > tile
    for A, B in cases:
        B = A if B is None else B
        Acp, Air = _dev(A.colptr, np.int64), _dev(A.rowidx, np.int32)
        Bcp, Bir = _dev(B.colptr, np.int64), _dev(B.rowidx, np.int32)
        out = torch.full((B.n + 1,), -7, dtype=torch.int64, device="cuda")
        stream.wait_stream(torch.cuda.current_stream())
        st = s.spgemm_colptr_noalloc(stream, A.m, A.n, B.n, Acp, Air, Bcp, Bir, out)
        assert st == 0
        dA = s.Matrix.csc(ctx, A.m, A.n, Acp, Air, _dev(A.vals, np.float64), PT_F64)
        dB = s.Matrix.csc(ctx, B.m, B.n, Bcp, Bir, _dev(B.vals, np.float64), PT_F64)
        ref = s.spgemm_multiply(ctx, dA, dB, PT_F64).export()[3]
        stream.synchronize()
        assert torch.equal(out, ref)
        want = np.zeros(B.n + 1, np.int64)
        np.cumsum(oracle.symbolic(A, B), out=want[1:])
        np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_colptr_noalloc_tall_and_wide_limits_against_oracle():
    """The two shapes that reach the entry point's other code paths: a column space
    of about 400k rows (the row bitmap needs more than 48 KiB of shared memory) and
    about 4.3 million columns (more than 1024 scan tiles), each against the oracle."""
    s = sp()
    stream = torch.cuda.Stream()
    tall_a = gen.erdos_renyi(400_000, 64, 50, 0x2204)
    tall_b = gen.erdos_renyi(64, 40, 6, 0x2205)
    wide_a = gen.erdos_renyi(64, 64, 3, 0x2206)
    wide_b = gen.erdos_renyi(64, 4_300_000, 1, 0x2207)
    for A, B in ((tall_a, tall_b), (wide_a, wide_b)):
        Acp, Air = _dev(A.colptr, np.int64), _dev(A.rowidx, np.int32)
        Bcp, Bir = _dev(B.colptr, np.int64), _dev(B.rowidx, np.int32)
        out = torch.full((B.n + 1,), -7, dtype=torch.int64, device="cuda")
        stream.wait_stream(torch.cuda.current_stream())
        assert s.spgemm_colptr_noalloc(stream, A.m, A.n, B.n, Acp, Air, Bcp, Bir, out) == 0
        stream.synchronize()
        want = np.zeros(B.n + 1, np.int64)
        np.cumsum(oracle.symbolic(A, B), out=want[1:])
        np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_colptr_noalloc_refuses_sizes_beyond_its_limits():
    s = sp()
    stream = torch.cuda.Stream()
    z = torch.zeros(2, dtype=torch.int64, device="cuda")
    r = torch.zeros(1, dtype=torch.int32, device="cuda")
    too_tall = 1048576 + 1                      # bitmap of m bits must fit shared memory
    assert s.spgemm_colptr_noalloc(stream, too_tall, 1, 1, z, r, z, r, z) == 8
    too_wide = 4096 * 4096 + 1                  # scan partials must fit the static scratch
    assert s.spgemm_colptr_noalloc(stream, 1, 1, too_wide, z, r, z, r, z) == 8
    assert s.spgemm_colptr_noalloc(stream, -1, 1, 1, z, r, z, r, z) == 1
