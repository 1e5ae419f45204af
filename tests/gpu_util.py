"""Helpers shared by the GPU parity tests (compare the CUDA path with the oracle)."""
from __future__ import annotations

import numpy as np

import oracle
from helpers import FP64_RTOL, PT_F64

_lib_built = False


def sp():
    """The binding, with the library built first (on the box it is built from source)."""
    global _lib_built
    if not _lib_built:
        from paper_1006_2183_gb300 import build
        build.build()
        _lib_built = True
    from paper_1006_2183_gb300 import spgemm
    return spgemm


def assert_matches(C, R, sr, rtol=FP64_RTOL, what=""):
    """C (binding HostCSC) vs R (oracle): structure bit-exact, values per the semiring contract."""
    assert (C.m, C.n) == (R.m, R.n), what
    np.testing.assert_array_equal(np.asarray(C.colptr), np.asarray(R.colptr), err_msg=f"colptr {what}")
    np.testing.assert_array_equal(np.asarray(C.rowidx), np.asarray(R.rowidx), err_msg=f"rowidx {what}")
    cv, rv = np.asarray(C.vals), np.asarray(R.vals)
    if sr == PT_F64:
        err = np.abs(cv - rv)
        bad = err > rtol * np.abs(rv)
        if bad.any():
            i = int(np.nonzero(bad)[0][0])
            raise AssertionError(f"{bad.sum()} values beyond rtol {rtol} {what}: first at {i}: {cv[i]} vs {rv[i]}")
    else:
        np.testing.assert_array_equal(cv, rv, err_msg=f"values {what}")


def gpu_product(ctx, A, B, sr, opts=None):
    s = sp()
    dA = s.Matrix.from_host(ctx, A, sr)
    dB = dA if B is A else s.Matrix.from_host(ctx, B, sr)
    return s.spgemm_multiply(ctx, dA, dB, sr, opts).to_host()


def check_product(ctx, A, B, sr, opts=None, what=""):
    C = gpu_product(ctx, A, B, sr, opts)
    R = oracle.spgemm(A, B, sr)
    assert_matches(C, R, sr, what=what)
    return C


def device_columns(C, cols):
    """Full column pointers and the sampled columns of a device result, gathered on the
    device so that products of tens of GB need not come to the host."""
    import torch
    m, n, nnz, cp, ir, v = C.export()
    torch.cuda.current_stream().wait_stream(C.ctx.stream)
    cols_t = torch.as_tensor(np.asarray(cols, dtype=np.int64), device=cp.device)
    start, end = cp[cols_t], cp[cols_t + 1]
    lens = end - start
    idx = torch.repeat_interleave(start, lens) + (torch.arange(int(lens.sum().item()), device=cp.device)
                                                   - torch.repeat_interleave(torch.cumsum(lens, 0) - lens, lens))
    sub_cp = np.zeros(len(cols) + 1, dtype=np.int64)
    np.cumsum(lens.cpu().numpy(), out=sub_cp[1:])
    return cp.cpu().numpy(), sub_cp, ir[idx].cpu().numpy(), v[idx].cpu().numpy()


def assert_sampled(C, A, B, sr, cols, what=""):
    """Sampled columns of a device product C = A*B against the oracle's columns."""
    cp, sub_cp, rows, vals = device_columns(C, cols)
    R = oracle.spgemm_columns(A, B, sr, np.asarray(cols, dtype=np.int64))
    np.testing.assert_array_equal(sub_cp, R.colptr, err_msg=f"sampled column lengths {what}")
    np.testing.assert_array_equal(rows, R.rowidx, err_msg=f"sampled rows {what}")
    if sr == PT_F64:
        bad = np.abs(vals - R.vals) > FP64_RTOL * np.abs(R.vals)
        assert not bad.any(), f"{bad.sum()} sampled values beyond rtol {what}"
    else:
        np.testing.assert_array_equal(vals, R.vals, err_msg=f"sampled values {what}")
    return cp
