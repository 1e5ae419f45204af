"""ctypes binding of libspgemm.so (argument marshalling only).

Every step of the product runs in the CUDA library; this module converts
torch tensors to device pointers, passes torch's current CUDA stream and
caching allocator to the library, and wraps library-owned outputs as
zero-copy torch views.  Importing it loads libspgemm.so and raises if the
library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspgemm.so")

PLUS_TIMES_F64, MIN_PLUS_F32, OR_AND_BOOL, PLUS_TIMES_I64 = 0, 1, 2, 3
FMT_CSC, FMT_CSR, FMT_DCSC = 0, 1, 2
TORCH_DTYPE = {PLUS_TIMES_F64: torch.float64, MIN_PLUS_F32: torch.float32, OR_AND_BOOL: torch.uint8,
               PLUS_TIMES_I64: torch.int64}
NP_DTYPE = {PLUS_TIMES_F64: np.float64, MIN_PLUS_F32: np.float32, OR_AND_BOOL: np.uint8, PLUS_TIMES_I64: np.int64}
TYPESTR = {PLUS_TIMES_F64: "<f8", MIN_PLUS_F32: "<f4", OR_AND_BOOL: "|u1", PLUS_TIMES_I64: "<i8"}
NPARAM = 1377
NPHASE = 8
NGROUP = 4
PHASES = ["analyze", "symbolic_hash", "symbolic_dense", "scan", "numeric_hash", "numeric_dense", "predict", "merge"]
STATUS = ["ok", "invalid argument", "dimension mismatch", "bad format", "out of memory", "index overflow",
          "timeout", "cuda error", "unsupported", "bad call order"]


class SpGEMMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS[status] if 0 <= status < len(STATUS) else status}: {msg}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libspgemm.so is not built ({LIB_PATH}); run __graft_entry__.build()")
_lib = ctypes.CDLL(LIB_PATH)

P = ctypes.c_void_p
I64 = ctypes.c_int64
PP = ctypes.POINTER(ctypes.c_void_p)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Opts(ctypes.Structure):
    _fields_ = [("use_predictor", ctypes.c_int), ("summa_fused", ctypes.c_int),
                ("summa_merge_every", ctypes.c_int), ("warp_max_flops", ctypes.c_int),
                ("block_max_flops", ctypes.c_int), ("dense_part_flops", ctypes.c_int),
                ("predictor_margin", ctypes.c_float), ("range_table_slots", ctypes.c_int),
                ("block_kernel", ctypes.c_int), ("range_slab_rows", ctypes.c_int),
                ("check_inputs", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


def _sig(name, args, res=ctypes.c_int):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_sig("spgemm_opts_default", [ctypes.POINTER(Opts)], None)
_sig("spgemm_ctx_create", [PP, P, ALLOC_FN, FREE_FN, P])
_sig("spgemm_ctx_destroy", [P])
_sig("spgemm_ctx_set_stream", [P, P])
_sig("spgemm_last_error", [P], ctypes.c_char_p)
_sig("spgemm_mat_csc", [P, PP, I64, I64, I64, P, P, P, ctypes.c_int])
_sig("spgemm_mat_csr", [P, PP, I64, I64, I64, P, P, P, ctypes.c_int])
_sig("spgemm_mat_validate", [P])
_sig("spgemm_mat_to_dcsc", [P, P, ctypes.c_int, PP])
_sig("spgemm_mat_transpose", [P, P, PP])
_sig("spgemm_mat_permute", [P, P, P, P, PP])
_sig("spgemm_summa_block_flops", [P, P, P, ctypes.c_int, ctypes.POINTER(I64)])
_sig("spgemm_mat_export", [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64), PP, PP, PP])
_sig("spgemm_mat_export_dcsc", [P, ctypes.POINTER(I64), PP, PP, ctypes.POINTER(I64), ctypes.POINTER(I64)])
_sig("spgemm_mat_format", [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)])
_sig("spgemm_mat_destroy", [P])
_sig("spgemm_plan", [P, P, P, ctypes.c_int, ctypes.POINTER(Opts), PP])
_sig("spgemm_symbolic", [P, ctypes.POINTER(I64)])
_sig("spgemm_numeric", [P, PP])
_sig("spgemm_plan_stats", [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)])
_sig("spgemm_plan_destroy", [P])
_sig("spgemm_multiply", [P, P, P, ctypes.c_int, ctypes.POINTER(Opts), PP])
_sig("spgemm_summa_blocked", [P, P, P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Opts), PP])
_sig("spgemm_summa_pipelined", [P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Opts), PP])
_sig("spgemm_summa_stats", [P, ctypes.POINTER(I64), ctypes.c_int, ctypes.POINTER(I64)])
_sig("spgemm_batch", [P, ctypes.c_int, PP, PP, ctypes.c_int, ctypes.POINTER(Opts), PP])
_sig("spgemm_batch_plan", [P, ctypes.c_int, PP, PP, ctypes.c_int, ctypes.POINTER(Opts), PP])
_sig("spgemm_batch_execute", [P])
_sig("spgemm_batch_outputs", [P, PP])
_sig("spgemm_autotune", [P, ctypes.c_int, PP, PP, ctypes.c_int, ctypes.POINTER(Opts)])
_sig("spgemm_colptr_noalloc", [P, I64, I64, I64, P, P, P, P, P])
_sig("spgemm_ctx_timing", [P, ctypes.c_int])
_sig("spgemm_ctx_phase_ms", [P, P, P])
_sig("spgemm_ctx_timing_group", [P, ctypes.c_int])
_sig("spgemm_launch_count", [], I64)
_sig("spgemm_plan_tier_stats", [P, P, P, P, P])
_sig("spgemm_predictor_set", [P, P])
_sig("spgemm_predictor_get", [P, P])
_sig("spgemm_predictor_features", [P, P, P, P, P])
_sig("spgemm_predictor_train_step", [P, P, P, I64, ctypes.c_float, P, P])
_sig("spgemm_predictor_forward", [P, P, I64, P])

EXPORTED = [n for n in dir(_lib) if n.startswith("spgemm_")]


def launch_count() -> int:
    """Kernels launched by libspgemm.so in this process so far."""
    return int(_lib.spgemm_launch_count())


def default_opts(**kw) -> Opts:
    o = Opts()
    _lib.spgemm_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return t.data_ptr()


class _CAI:
    """Zero-copy description of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr or 0, False),
                                         "version": 3, "strides": None}


def _view(ptr: int | None, n: int, typestr: str, dtype: torch.dtype, device) -> torch.Tensor:
    if n == 0 or not ptr:
        return torch.empty(0, dtype=dtype, device=device)
    return torch.as_tensor(_CAI(ptr, n, typestr), device=device)


def _order_after_current(ctx):
    """Work the caller queued on torch's current stream (e.g. uploads) precedes the library's."""
    cur = torch.cuda.current_stream()
    if cur.cuda_stream != ctx.stream.cuda_stream:
        ctx.stream.wait_stream(cur)


class Context:
    """Library context bound to a CUDA stream; device memory comes from torch's caching allocator."""

    def __init__(self, stream: torch.cuda.Stream | None = None, torch_allocator: bool = True):
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream or torch.cuda.current_stream()
        self._h = ctypes.c_void_p()
        if torch_allocator:
            dev = self.device.index
            tstream = self.stream

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, tstream)
                except Exception:
                    return None

            def _free(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
        else:
            self._alloc_cb = ALLOC_FN()
            self._free_cb = FREE_FN()
        self._check(_lib.spgemm_ctx_create(ctypes.byref(self._h), ctypes.c_void_p(self.stream.cuda_stream),
                                           self._alloc_cb, self._free_cb, None))

    def _check(self, st: int):
        if st != 0:
            msg = _lib.spgemm_last_error(self._h).decode() if self._h else ""
            raise SpGEMMError(st, msg)

    @property
    def handle(self):
        return self._h

    def timing(self, enable: bool):
        self._check(_lib.spgemm_ctx_timing(self._h, int(enable)))

    def timing_group(self, group: int):
        self._check(_lib.spgemm_ctx_timing_group(self._h, group))

    def phase_ms(self) -> dict:
        """{(group, semiring, phase name): (total ms, count)} since timing was enabled."""
        n = NGROUP * 4 * NPHASE
        ms = (ctypes.c_double * n)()
        cnt = (I64 * n)()
        self._check(_lib.spgemm_ctx_phase_ms(self._h, ms, cnt))
        return {(g, sr, PHASES[i]): (ms[(g * 4 + sr) * NPHASE + i], cnt[(g * 4 + sr) * NPHASE + i])
                for g in range(NGROUP) for sr in range(4) for i in range(NPHASE)}

    def close(self):
        if self._h:
            _lib.spgemm_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Matrix:
    """A library matrix handle.  Borrowed handles keep their torch tensors alive."""

    def __init__(self, ctx: Context, handle: ctypes.c_void_p, semiring: int, keep=()):
        self.ctx = ctx
        self._h = handle
        self.semiring = semiring
        self._keep = list(keep)

    @classmethod
    def csc(cls, ctx: Context, m: int, n: int, colptr: torch.Tensor, rowidx: torch.Tensor,
            vals: torch.Tensor | None, semiring: int) -> "Matrix":
        h = ctypes.c_void_p()
        nnz = int(rowidx.numel())
        _order_after_current(ctx)
        ctx._check(_lib.spgemm_mat_csc(ctx.handle, ctypes.byref(h), m, n, nnz, _ptr(colptr), _ptr(rowidx),
                                       _ptr(vals), semiring))
        return cls(ctx, h, semiring, (colptr, rowidx, vals))

    @classmethod
    def csr(cls, ctx: Context, m: int, n: int, rowptr: torch.Tensor, colidx: torch.Tensor,
            vals: torch.Tensor | None, semiring: int) -> "Matrix":
        h = ctypes.c_void_p()
        _order_after_current(ctx)
        ctx._check(_lib.spgemm_mat_csr(ctx.handle, ctypes.byref(h), m, n, int(colidx.numel()), _ptr(rowptr),
                                       _ptr(colidx), _ptr(vals), semiring))
        return cls(ctx, h, semiring, (rowptr, colidx, vals))

    @classmethod
    def from_host(cls, ctx: Context, A, semiring: int) -> "Matrix":
        """Upload a host CSC (attributes m, n, colptr, rowidx, vals) into torch device tensors."""
        dev = ctx.device
        cp = torch.from_numpy(np.ascontiguousarray(A.colptr, np.int64)).to(dev)
        ir = torch.from_numpy(np.ascontiguousarray(A.rowidx, np.int32)).to(dev)
        v = torch.from_numpy(np.ascontiguousarray(A.vals, NP_DTYPE[semiring])).to(dev)
        return cls.csc(ctx, A.m, A.n, cp, ir, v, semiring)

    @property
    def handle(self):
        return self._h

    def shape(self):
        m, n, nnz = I64(), I64(), I64()
        self.ctx._check(_lib.spgemm_mat_export(self._h, ctypes.byref(m), ctypes.byref(n), ctypes.byref(nnz),
                                               None, None, None))
        return m.value, n.value, nnz.value

    def format(self) -> int:
        f, s = ctypes.c_int(), ctypes.c_int()
        self.ctx._check(_lib.spgemm_mat_format(self._h, ctypes.byref(f), ctypes.byref(s)))
        return f.value

    def export(self):
        """(m, n, nnz, colptr, rowidx, vals) with zero-copy device views (CP for DCSC)."""
        m, n, nnz = I64(), I64(), I64()
        cp, ir, v = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        self.ctx._check(_lib.spgemm_mat_export(self._h, ctypes.byref(m), ctypes.byref(n), ctypes.byref(nnz),
                                               ctypes.byref(cp), ctypes.byref(ir), ctypes.byref(v)))
        dev = self.ctx.device
        fmt = self.format()
        if fmt == FMT_DCSC:
            nzc = I64()
            self.ctx._check(_lib.spgemm_mat_export_dcsc(self._h, ctypes.byref(nzc), None, None, None, None))
            ncp = nzc.value + 1
        elif fmt == FMT_CSR:
            ncp = m.value + 1
        else:
            ncp = n.value + 1
        return (m.value, n.value, nnz.value, _view(cp.value, ncp, "<i8", torch.int64, dev),
                _view(ir.value, nnz.value, "<i4", torch.int32, dev),
                _view(v.value, nnz.value, TYPESTR[self.semiring], TORCH_DTYPE[self.semiring], dev))

    def export_dcsc(self):
        nzc, naux, chunk = I64(), I64(), I64()
        jc, aux = ctypes.c_void_p(), ctypes.c_void_p()
        self.ctx._check(_lib.spgemm_mat_export_dcsc(self._h, ctypes.byref(nzc), ctypes.byref(jc), ctypes.byref(aux),
                                                    ctypes.byref(naux), ctypes.byref(chunk)))
        dev = self.ctx.device
        auxv = _view(aux.value, naux.value + 1, "<i4", torch.int32, dev) if aux.value else None
        return nzc.value, _view(jc.value, nzc.value, "<i4", torch.int32, dev), auxv, chunk.value

    def to_host(self):
        """Copy to a host CSC (numpy arrays); synchronises the context stream."""
        m, n, nnz, cp, ir, v = self.export()
        torch.cuda.current_stream().wait_stream(self.ctx.stream)
        return HostCSC(m, n, cp.cpu().numpy(), ir.cpu().numpy(), v.cpu().numpy())

    def validate(self):
        self.ctx._check(_lib.spgemm_mat_validate(self._h))

    def close(self):
        if self._h:
            _lib.spgemm_mat_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class HostCSC:
    m: int
    n: int
    colptr: np.ndarray
    rowidx: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self):
        return int(self.colptr[-1])


class Plan:
    def __init__(self, ctx: Context, handle, A: Matrix, B: Matrix, semiring: int):
        self.ctx, self._h, self.A, self.B, self.semiring = ctx, handle, A, B, semiring

    def stats(self):
        fl, nz, ov = I64(), I64(), I64()
        tiers = (I64 * 4)()
        self.ctx._check(_lib.spgemm_plan_stats(self._h, ctypes.byref(fl), ctypes.byref(nz), tiers, ctypes.byref(ov)))
        return {"flops": fl.value, "nnz": nz.value, "tiers": list(tiers), "overflow_cols": ov.value}

    def tier_stats(self):
        cols, fl, nz, bn = (I64 * 4)(), (I64 * 4)(), (I64 * 4)(), (I64 * 4)()
        self.ctx._check(_lib.spgemm_plan_tier_stats(self._h, cols, fl, nz, bn))
        return {"cols": list(cols), "flops": list(fl), "nnz": list(nz), "bnnz": list(bn)}

    def close(self):
        if self._h:
            _lib.spgemm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- C-ABI functions by name
def _opts(o):
    return ctypes.byref(o) if o is not None else None


def spgemm_plan(ctx: Context, A: Matrix, B: Matrix, semiring: int, opts: Opts | None = None) -> Plan:
    h = ctypes.c_void_p()
    ctx._check(_lib.spgemm_plan(ctx.handle, A.handle, B.handle, semiring, _opts(opts), ctypes.byref(h)))
    return Plan(ctx, h, A, B, semiring)


def spgemm_symbolic(plan: Plan) -> int:
    nnz = I64()
    plan.ctx._check(_lib.spgemm_symbolic(plan._h, ctypes.byref(nnz)))
    return nnz.value


def spgemm_numeric(plan: Plan) -> Matrix:
    h = ctypes.c_void_p()
    plan.ctx._check(_lib.spgemm_numeric(plan._h, ctypes.byref(h)))
    return Matrix(plan.ctx, h, plan.semiring)


def spgemm_multiply(ctx: Context, A: Matrix, B: Matrix, semiring: int, opts: Opts | None = None) -> Matrix:
    h = ctypes.c_void_p()
    ctx._check(_lib.spgemm_multiply(ctx.handle, A.handle, B.handle, semiring, _opts(opts), ctypes.byref(h)))
    return Matrix(ctx, h, semiring)


def spgemm_summa_blocked(ctx: Context, A: Matrix, B: Matrix, g: int, semiring: int,
                         opts: Opts | None = None) -> Matrix:
    h = ctypes.c_void_p()
    ctx._check(_lib.spgemm_summa_blocked(ctx.handle, A.handle, B.handle, g, semiring, _opts(opts), ctypes.byref(h)))
    return Matrix(ctx, h, semiring)


def spgemm_summa_pipelined(ctx: Context, merge_ctx: Context, A: Matrix, B: Matrix, g: int, semiring: int,
                           opts: Opts | None = None) -> Matrix:
    """spgemm_summa_blocked with the stage merges on merge_ctx's stream; C belongs to merge_ctx."""
    h = ctypes.c_void_p()
    _order_after_current(ctx)
    ctx._check(_lib.spgemm_summa_pipelined(ctx.handle, merge_ctx.handle, A.handle, B.handle, g, semiring,
                                           _opts(opts), ctypes.byref(h)))
    return Matrix(merge_ctx, h, semiring)


def spgemm_summa_stats(ctx: Context, g: int):
    sf = (I64 * g)()
    ne = I64()
    ctx._check(_lib.spgemm_summa_stats(ctx.handle, sf, g, ctypes.byref(ne)))
    return list(sf), ne.value


def spgemm_batch(ctx: Context, As: list[Matrix], Bs: list[Matrix], semiring: int,
                 opts: Opts | None = None) -> list[Matrix]:
    n = len(As)
    ah = (ctypes.c_void_p * n)(*[a.handle.value for a in As])
    bh = (ctypes.c_void_p * n)(*[b.handle.value for b in Bs])
    ch = (ctypes.c_void_p * n)()
    ctx._check(_lib.spgemm_batch(ctx.handle, n, ah, bh, semiring, _opts(opts), ch))
    return [Matrix(ctx, ctypes.c_void_p(ch[i]), semiring) for i in range(n)]


def _handles(ms):
    return (ctypes.c_void_p * len(ms))(*[m.handle.value for m in ms])


class BatchPlan(Plan):
    """Batch plan: analysis and symbolic pass done once; execute() recomputes values (CUDA graph replay)."""

    def __init__(self, ctx, handle, As, Bs, semiring):
        super().__init__(ctx, handle, None, None, semiring)
        self._keep = (list(As), list(Bs))
        self.count = len(As)

    def execute(self):
        self.ctx._check(_lib.spgemm_batch_execute(self._h))

    def outputs(self) -> list[Matrix]:
        ch = (ctypes.c_void_p * self.count)()
        self.ctx._check(_lib.spgemm_batch_outputs(self._h, ch))
        return [Matrix(self.ctx, ctypes.c_void_p(ch[i]), self.semiring, (self,)) for i in range(self.count)]


def spgemm_batch_plan(ctx: Context, As: list[Matrix], Bs: list[Matrix], semiring: int,
                      opts: Opts | None = None) -> BatchPlan:
    h = ctypes.c_void_p()
    ctx._check(_lib.spgemm_batch_plan(ctx.handle, len(As), _handles(As), _handles(Bs), semiring, _opts(opts),
                                      ctypes.byref(h)))
    return BatchPlan(ctx, h, As, Bs, semiring)


def spgemm_autotune(ctx: Context, As: list[Matrix], Bs: list[Matrix], semiring: int,
                    opts: Opts | None = None) -> Opts:
    o = opts if opts is not None else default_opts()
    ctx._check(_lib.spgemm_autotune(ctx.handle, len(As), _handles(As), _handles(Bs), semiring, ctypes.byref(o)))
    return o


def spgemm_colptr_noalloc(stream: torch.cuda.Stream, m: int, k: int, n: int, Acolptr: torch.Tensor,
                          Arowidx: torch.Tensor, Bcolptr: torch.Tensor, Browidx: torch.Tensor,
                          Ccolptr: torch.Tensor) -> int:
    """C's column pointers into Ccolptr (n+1 int64, device) without any device allocation.

    Returns the library status (0 on success); nothing is allocated by the
    library or by this wrapper.
    """
    return int(_lib.spgemm_colptr_noalloc(ctypes.c_void_p(stream.cuda_stream), m, k, n, _ptr(Acolptr),
                                          _ptr(Arowidx), _ptr(Bcolptr), _ptr(Browidx), _ptr(Ccolptr)))


def spgemm_mat_to_dcsc(ctx: Context, A: Matrix, build_aux: bool = True) -> Matrix:
    h = ctypes.c_void_p()
    ctx._check(_lib.spgemm_mat_to_dcsc(ctx.handle, A.handle, int(build_aux), ctypes.byref(h)))
    return Matrix(ctx, h, A.semiring, (A,))


def spgemm_mat_permute(ctx: Context, A: Matrix, row_perm: torch.Tensor | None = None,
                       col_perm: torch.Tensor | None = None) -> Matrix:
    """B = P A Q^T with B(row_perm[i], col_perm[j]) = A(i, j); perms are device int32 tensors."""
    for t in (row_perm, col_perm):
        if t is not None:
            assert t.dtype == torch.int32 and t.is_cuda and t.is_contiguous()
    _order_after_current(ctx)
    h = ctypes.c_void_p()
    ctx._check(_lib.spgemm_mat_permute(ctx.handle, A.handle, _ptr(row_perm), _ptr(col_perm), ctypes.byref(h)))
    return Matrix(ctx, h, A.semiring, (A,))


def spgemm_summa_block_flops(ctx: Context, A: Matrix, B: Matrix, g: int) -> np.ndarray:
    """flops of every block product of the g x g grid, as an array indexed [s, J, I]."""
    out = (I64 * (g * g * g))()
    _order_after_current(ctx)
    ctx._check(_lib.spgemm_summa_block_flops(ctx.handle, A.handle, B.handle, g, out))
    return np.frombuffer(out, dtype=np.int64).reshape(g, g, g).copy()


def spgemm_mat_transpose(ctx: Context, A: Matrix) -> Matrix:
    h = ctypes.c_void_p()
    ctx._check(_lib.spgemm_mat_transpose(ctx.handle, A.handle, ctypes.byref(h)))
    return Matrix(ctx, h, A.semiring, (A,))


def spgemm_predictor_set(ctx: Context, params: np.ndarray):
    p = np.ascontiguousarray(params, np.float32)
    assert p.size == NPARAM
    ctx._check(_lib.spgemm_predictor_set(ctx.handle, p.ctypes.data_as(ctypes.c_void_p)))


def spgemm_predictor_get(ctx: Context) -> np.ndarray:
    p = np.zeros(NPARAM, np.float32)
    ctx._check(_lib.spgemm_predictor_get(ctx.handle, p.ctypes.data_as(ctypes.c_void_p)))
    return p


def spgemm_predictor_features(ctx: Context, A: Matrix, B: Matrix, want_labels: bool = True):
    _, n, _ = B.shape()
    X = torch.empty((n, 8), dtype=torch.float32, device=ctx.device)
    y = torch.empty(n, dtype=torch.int64, device=ctx.device) if want_labels else None
    ctx._check(_lib.spgemm_predictor_features(ctx.handle, A.handle, B.handle, _ptr(X), _ptr(y)))
    return X, y


def spgemm_predictor_train_step(ctx: Context, X: torch.Tensor, y: torch.Tensor, lr: float, want_grad=False):
    loss = ctypes.c_float()
    g = np.zeros(NPARAM, np.float32) if want_grad else None
    ctx._check(_lib.spgemm_predictor_train_step(ctx.handle, _ptr(X), _ptr(y), int(X.shape[0]), lr,
                                                ctypes.byref(loss),
                                                g.ctypes.data_as(ctypes.c_void_p) if g is not None else None))
    return loss.value, g


def spgemm_predictor_forward(ctx: Context, X: torch.Tensor) -> torch.Tensor:
    out = torch.empty(X.shape[0], dtype=torch.float32, device=ctx.device)
    ctx._check(_lib.spgemm_predictor_forward(ctx.handle, _ptr(X), int(X.shape[0]), _ptr(out)))
    return out
