"""The library's own waits on the device read their few bytes (counts, offsets,
flags) through mapped pinned host memory written by a kernel, not with a
device-to-host copy, which would queue behind every bulk device-to-host copy
already on the copy engine.  Checked here: a product's host call returns while an
8 GiB copy back on another stream is still running, with a result equal to the
oracle's; and a batch whose per-product offsets (8 bytes each) outgrow the first
read-back buffer of the context is still exact.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import assert_matches, sp
from helpers import PT_F64, PT_I64
from paper_1006_2183_gb300 import gen

pytestmark = pytest.mark.gpu


def test_product_does_not_wait_for_a_bulk_copy_on_another_stream():
    s = sp()
    ctx = s.Context(stream=torch.cuda.Stream())
    A = gen.rmat(12, 8, 0x5300)
    dA = s.Matrix.from_host(ctx, A, PT_F64)
    s.spgemm_multiply(ctx, dA, dA, PT_F64)   # the first call loads the kernels
    big = torch.empty(8 << 30, dtype=torch.uint8, device="cuda")
    host = torch.empty(8 << 30, dtype=torch.uint8, pin_memory=True)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        host.copy_(big, non_blocking=True)   # well over 20 ms on any host link
        copied = torch.cuda.Event()
        copied.record(side)
    C = s.spgemm_multiply(ctx, dA, dA, PT_F64)   # waits on the device for C's size
    still_copying = not copied.query()
    side.synchronize()
    del big, host
    assert still_copying, "the product's waits on the device queued behind the bulk copy"
    assert_matches(C.to_host(), oracle.spgemm(A, A, PT_F64), PT_F64, what="product during the copy")


def test_batch_offsets_larger_than_the_first_read_back_buffer():
    s = sp()
    ctx = s.Context(stream=torch.cuda.Stream())
    n = 9000   # 8 * (n + 1) bytes of product offsets: more than the context's first 64 KiB
    B = gen.erdos_renyi(16, 12, 3, 0x5150, PT_I64)
    As = [gen.erdos_renyi(20, 16, 2, 0x5200 + i, PT_I64) for i in range(n)]
    dB = s.Matrix.from_host(ctx, B, PT_I64)
    Cs = s.spgemm_batch(ctx, [s.Matrix.from_host(ctx, a, PT_I64) for a in As], [dB] * n, PT_I64)
    assert len(Cs) == n
    for i in list(range(0, n, 97)) + [n - 1]:
        assert_matches(Cs[i].to_host(), oracle.spgemm(As[i], B, PT_I64), PT_I64, what=f"product {i}")
