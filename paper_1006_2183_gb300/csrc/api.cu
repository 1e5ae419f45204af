// C-ABI of the library: contexts, matrix handles, and the flat product
// (plan -> symbolic -> numeric).  Declarations and contracts: spgemm.h.
#include <algorithm>
#include <cstring>

#include "internal.cuh"

using namespace sg;

// ------------------------------------------------------------------ context / memory
spgemm_status_t set_err(spgemm_ctx* ctx, spgemm_status_t s, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return s;
}

spgemm_status_t check_cuda(spgemm_ctx* ctx, cudaError_t e, const char* what) {
    return set_err(ctx, SPGEMM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void* ctx_alloc(spgemm_ctx* ctx, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) / 256 * 256;
    if (ctx->alloc) return ctx->alloc(bytes, ctx->user);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void ctx_free(spgemm_ctx* ctx, void* p) {
    if (!p) return;
    if (ctx->free_fn) ctx->free_fn(p, ctx->user);
    else cudaFreeAsync(p, ctx->stream);
}

DevBuf::~DevBuf() { ctx_free(ctx, p); }

std::shared_ptr<DevBuf> ctx_buf(spgemm_ctx* ctx, size_t bytes) {
    void* p = ctx_alloc(ctx, bytes);
    if (!p) return nullptr;
    return std::make_shared<DevBuf>(ctx, p);
}

size_t sr_size(spgemm_semiring_t sr) {
    switch (sr) {
    case SPGEMM_PLUS_TIMES_F64: return 8;
    case SPGEMM_MIN_PLUS_F32: return 4;
    case SPGEMM_OR_AND_BOOL: return 1;
    case SPGEMM_PLUS_TIMES_I64: return 8;
    }
    return 0;
}

spgemm_status_t sync_ctx(spgemm_ctx* ctx) {
    SG_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    SG_CUDA(ctx, cudaGetLastError());
    return SPGEMM_OK;
}

DMat dmat_of(const spgemm_mat* M) {
    DMat d;
    d.m = M->m;
    d.n = M->n;
    d.nnz = M->nnz;
    d.cp = M->cp;
    d.ir = M->ir;
    d.num = M->num;
    if (M->fmt == SPGEMM_FMT_DCSC) {
        d.nzc = M->nzc;
        d.jc = M->jc;
        d.aux = M->aux;
        d.naux = M->naux;
        d.chunk = M->chunk;
    } else {
        d.nzc = M->n;
    }
    return d;
}

extern "C" {

const char* spgemm_status_string(spgemm_status_t s) {
    switch (s) {
    case SPGEMM_OK: return "ok";
    case SPGEMM_ERR_INVALID_ARG: return "invalid argument";
    case SPGEMM_ERR_DIM_MISMATCH: return "dimension mismatch";
    case SPGEMM_ERR_BAD_FORMAT: return "bad format";
    case SPGEMM_ERR_OOM: return "out of memory";
    case SPGEMM_ERR_INDEX_OVERFLOW: return "index overflow";
    case SPGEMM_ERR_TIMEOUT: return "timeout";
    case SPGEMM_ERR_CUDA: return "cuda error";
    case SPGEMM_ERR_UNSUPPORTED: return "unsupported";
    case SPGEMM_ERR_STATE: return "bad call order";
    }
    return "unknown";
}

void spgemm_opts_default(spgemm_opts_t* o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->use_predictor = 0;
    o->summa_fused = 0;
    o->summa_merge_every = 0;
    o->warp_max_flops = 512;
    o->block_max_flops = 4096;
    o->dense_part_flops = 65536;
    o->predictor_margin = 0.25f;
}

spgemm_status_t spgemm_ctx_create(spgemm_ctx_t* out, void* stream, spgemm_alloc_fn alloc, spgemm_free_fn free_fn,
                                  void* user) {
    if (!out) return SPGEMM_ERR_INVALID_ARG;
    if ((alloc == nullptr) != (free_fn == nullptr)) return SPGEMM_ERR_INVALID_ARG;
    auto* c = new spgemm_ctx();
    c->stream = (cudaStream_t)stream;
    c->alloc = alloc;
    c->free_fn = free_fn;
    c->user = user;
    cudaGetDevice(&c->device);
    *out = c;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_ctx_set_stream(spgemm_ctx_t ctx, void* stream) {
    if (!ctx) return SPGEMM_ERR_INVALID_ARG;
    ctx->stream = (cudaStream_t)stream;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_ctx_destroy(spgemm_ctx_t ctx) {
    if (!ctx) return SPGEMM_ERR_INVALID_ARG;
    ctx_free(ctx, ctx->pred);
    ctx_free(ctx, ctx->adam_m);
    ctx_free(ctx, ctx->adam_v);
    ctx_free(ctx, ctx->grad);
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
    return SPGEMM_OK;
}

const char* spgemm_last_error(spgemm_ctx_t ctx) { return ctx ? ctx->err.c_str() : "null context"; }

// ------------------------------------------------------------------ matrices
static spgemm_status_t check_sr(spgemm_ctx* ctx, spgemm_semiring_t sr) {
    if ((int)sr < 0 || (int)sr > 3) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "bad semiring %d", (int)sr);
    return SPGEMM_OK;
}

spgemm_status_t spgemm_mat_csc(spgemm_ctx_t ctx, spgemm_mat_t* out, int64_t m, int64_t n, int64_t nnz,
                               const int64_t* colptr, const int32_t* rowidx, const void* vals,
                               spgemm_semiring_t sr) {
    if (!ctx || !out) return SPGEMM_ERR_INVALID_ARG;
    SG_TRY(check_sr(ctx, sr));
    if (m < 0 || n < 0 || nnz < 0) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "negative size");
    if (m > INT32_MAX) return set_err(ctx, SPGEMM_ERR_INDEX_OVERFLOW, "m = %lld exceeds int32 rows", (long long)m);
    if (n > INT32_MAX) return set_err(ctx, SPGEMM_ERR_INDEX_OVERFLOW, "n too large");
    if (!colptr || (nnz > 0 && !rowidx)) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "null array");
    auto* M = new spgemm_mat();
    M->ctx = ctx;
    M->fmt = SPGEMM_FMT_CSC;
    M->sr = sr;
    M->m = m;
    M->n = n;
    M->nnz = nnz;
    M->cp = colptr;
    M->ir = rowidx;
    M->num = vals;
    M->nzc = n;
    *out = M;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_mat_csr(spgemm_ctx_t ctx, spgemm_mat_t* out, int64_t m, int64_t n, int64_t nnz,
                               const int64_t* rowptr, const int32_t* colidx, const void* vals,
                               spgemm_semiring_t sr) {
    // a CSR m x n matrix is stored exactly like the CSC of its n x m transpose
    SG_TRY(spgemm_mat_csc(ctx, out, n, m, nnz, rowptr, colidx, vals, sr));
    (*out)->fmt = SPGEMM_FMT_CSR;
    (*out)->m = m;
    (*out)->n = n;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_mat_export(spgemm_mat_t M, int64_t* m, int64_t* n, int64_t* nnz, const int64_t** colptr,
                                  const int32_t** rowidx, const void** vals) {
    if (!M) return SPGEMM_ERR_INVALID_ARG;
    if (m) *m = M->m;
    if (n) *n = M->n;
    if (nnz) *nnz = M->nnz;
    if (colptr) *colptr = M->cp;
    if (rowidx) *rowidx = M->ir;
    if (vals) *vals = M->num;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_mat_export_dcsc(spgemm_mat_t M, int64_t* nzc, const int32_t** jc, const int32_t** aux,
                                       int64_t* naux, int64_t* chunk) {
    if (!M) return SPGEMM_ERR_INVALID_ARG;
    if (M->fmt != SPGEMM_FMT_DCSC) return set_err(M->ctx, SPGEMM_ERR_INVALID_ARG, "not a DCSC handle");
    if (nzc) *nzc = M->nzc;
    if (jc) *jc = M->jc;
    if (aux) *aux = M->aux;
    if (naux) *naux = M->naux;
    if (chunk) *chunk = M->chunk;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_mat_format(spgemm_mat_t M, spgemm_format_t* fmt, spgemm_semiring_t* sr) {
    if (!M) return SPGEMM_ERR_INVALID_ARG;
    if (fmt) *fmt = M->fmt;
    if (sr) *sr = M->sr;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_mat_destroy(spgemm_mat_t M) {
    if (!M) return SPGEMM_ERR_INVALID_ARG;
    delete M;
    return SPGEMM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ plan
static spgemm_status_t to_csc_operand(spgemm_ctx* ctx, spgemm_mat_t M, spgemm_mat_t* conv, DMat* d) {
    if (M->fmt == SPGEMM_FMT_CSR) {
        // stored arrays are the CSC of M^T (n x m); transposing them gives M's CSC
        spgemm_mat_t T = new spgemm_mat();
        spgemm_status_t s = transpose_csc(ctx, M->n, M->m, M->nnz, M->cp, M->ir, M->num, sr_size(M->sr), T);
        if (s != SPGEMM_OK) {
            delete T;
            return s;
        }
        T->sr = M->sr;
        *conv = T;
        *d = dmat_of(T);
        return SPGEMM_OK;
    }
    *d = dmat_of(M);
    return SPGEMM_OK;
}

spgemm_status_t plan_build(spgemm_ctx* ctx, const DMat& A, const DMat& B, spgemm_semiring_t sr,
                           const spgemm_opts_t& opts, struct spgemm_plan* P) {
    P->ctx = ctx;
    P->sr = sr;
    P->opts = opts;
    P->A = A;
    P->B = B;
    P->m = A.m;
    P->n = B.n;
    P->cfg.warp_max = std::max(0, std::min(opts.warp_max_flops, 512));
    P->cfg.block_max = std::max(P->cfg.warp_max, std::min(opts.block_max_flops, 4096));
    P->cfg.dense_rows = dense_rows_for(sr, 0);
    P->cfg.part_flops = std::max(1024, opts.dense_part_flops);
    cudaStream_t st = ctx->stream;
    const int64_t nzcB = B.nzc;
    // one arena for the per-column arrays of the plan
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    size_t o_flops = take(8 * std::max<int64_t>(nzcB, 1));
    size_t o_bin = take(std::max<int64_t>(nzcB, 1));
    size_t o_ctr = take(8 * (2 * NBIN + 2));
    size_t o_binoff = take(8 * NBIN);
    size_t o_list = take(4 * std::max<int64_t>(nzcB, 1));
    size_t o_nnz = take(8 * std::max<int64_t>(B.n, 1));
    size_t o_scan = take(scan_tmp_bytes(B.n));
    size_t o_feat = opts.use_predictor ? take(32 * std::max<int64_t>(nzcB, 1)) : 0;
    size_t o_sk = opts.use_predictor ? take(8 * std::max<int64_t>(A.n, 1)) : 0;
    auto arena = ctx_buf(ctx, off);
    if (!arena) return set_err(ctx, SPGEMM_ERR_OOM, "plan arena of %zu bytes", off);
    P->bufs.push_back(arena);
    char* base = (char*)arena->p;
    P->flops = (int64_t*)(base + o_flops);
    P->bin = (uint8_t*)(base + o_bin);
    P->ctr = (unsigned long long*)(base + o_ctr);
    P->bin_off_dev = (int64_t*)(base + o_binoff);
    P->list = (int32_t*)(base + o_list);
    P->nnz_col = (int64_t*)(base + o_nnz);
    P->scan_tmp = base + o_scan;
    uint64_t* sketch = nullptr;
    if (opts.use_predictor) {
        P->feat = (float*)(base + o_feat);
        sketch = (uint64_t*)(base + o_sk);
        launch_row_sketch(st, A, sketch);
    }
    PhaseTimer t_an(ctx, SPGEMM_PHASE_ANALYZE, sr);
    SG_CUDA(ctx, cudaMemsetAsync(P->ctr, 0, 8 * (2 * NBIN + 2), st));
    launch_analyze(st, A, B, P->cfg, P->flops, P->bin, P->ctr, P->ctr + 2 * NBIN, sketch, P->feat);
    unsigned long long hc[NBIN + 1];
    SG_CUDA(ctx, cudaMemcpyAsync(hc, P->ctr, sizeof(unsigned long long) * NBIN, cudaMemcpyDeviceToHost, st));
    SG_CUDA(ctx, cudaMemcpyAsync(hc + NBIN, P->ctr + 2 * NBIN, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    SG_TRY(sync_ctx(ctx));
    int64_t acc = 0;
    for (int b = 0; b < NBIN; ++b) {
        P->bin_cnt[b] = (int64_t)hc[b];
        P->bin_off[b] = acc;
        acc += P->bin_cnt[b];
    }
    P->flops_total = (int64_t)hc[NBIN];
    SG_CUDA(ctx, cudaMemcpyAsync(P->bin_off_dev, P->bin_off, sizeof(int64_t) * NBIN, cudaMemcpyHostToDevice, st));
    launch_bin_scatter(st, nzcB, P->bin, P->bin_off_dev, P->ctr + NBIN, P->list);
    const int64_t nd = P->bin_cnt[BIN_DENSE];
    if (nd > 0) {
        P->G = ceil_div64(A.m, P->cfg.dense_rows);
        const int64_t maxp = std::min<int64_t>(P->G, MAX_PARTS);
        size_t o2 = 0;
        off = 0;
        size_t o_items = take(sizeof(int2) * nd * maxp);
        size_t o_np = take(nd);
        size_t o_pc = take(4 * nd * maxp);
        size_t o_cur = take(4 * std::max<int64_t>(B.nnz, 1) * maxp);
        (void)o2;
        auto dbuf = ctx_buf(ctx, off);
        if (!dbuf) return set_err(ctx, SPGEMM_ERR_OOM, "dense-tier arena of %zu bytes", off);
        P->bufs.push_back(dbuf);
        char* db = (char*)dbuf->p;
        P->items = (int2*)(db + o_items);
        P->nparts = (int8_t*)(db + o_np);
        P->part_count = (int32_t*)(db + o_pc);
        P->cursors = (int32_t*)(db + o_cur);
        launch_dense_items(st, P->list + P->bin_off[BIN_DENSE], nd, P->flops, (int)P->G, P->cfg.part_flops, P->items,
                           P->ctr + 2 * NBIN + 1, P->nparts);
    }
    SG_CUDA(ctx, cudaGetLastError());
    return SPGEMM_OK;
}

template <class SR>
static void dispatch_symbolic(struct spgemm_plan* P) {
    const int64_t nd = P->bin_cnt[BIN_DENSE];
    for (int which = 1; which <= 2; ++which) {
        PhaseTimer t(P->ctx, which == 1 ? SPGEMM_PHASE_SYMBOLIC_HASH : SPGEMM_PHASE_SYMBOLIC_DENSE, P->sr);
        launch_symbolic<SR>(P->ctx->stream, P->A, P->B, P->cfg, P->list, P->bin_off, P->bin_cnt, P->items,
                            P->ctr + 2 * NBIN + 1, nd * std::min<int64_t>(std::max<int64_t>(P->G, 1), MAX_PARTS),
                            P->nparts, P->cursors, P->part_count, P->nnz_col, which);
    }
}

template <class SR>
static void dispatch_numeric(struct spgemm_plan* P, int32_t* Cir, void* Cv) {
    const int64_t nd = P->bin_cnt[BIN_DENSE];
    for (int which = 1; which <= 2; ++which) {
        PhaseTimer t(P->ctx, which == 1 ? SPGEMM_PHASE_NUMERIC_HASH : SPGEMM_PHASE_NUMERIC_DENSE, P->sr);
        launch_numeric<SR>(P->ctx->stream, P->A, P->B, P->cfg, P->list, P->bin_off, P->bin_cnt, P->items,
                           P->ctr + 2 * NBIN + 1, nd * std::min<int64_t>(std::max<int64_t>(P->G, 1), MAX_PARTS),
                           P->cursors, P->part_count, P->nparts, P->Ccp, Cir, (typename SR::T*)Cv, which);
    }
}

static void run_symbolic_kernels(struct spgemm_plan* P) {
    cudaStream_t st = P->ctx->stream;
    cudaMemsetAsync(P->nnz_col, 0, 8 * std::max<int64_t>(P->n, 1), st);
    switch (P->sr) {
    case SPGEMM_PLUS_TIMES_F64: dispatch_symbolic<PT64>(P); break;
    case SPGEMM_MIN_PLUS_F32: dispatch_symbolic<MP32>(P); break;
    case SPGEMM_OR_AND_BOOL: dispatch_symbolic<BOOL8>(P); break;
    case SPGEMM_PLUS_TIMES_I64: dispatch_symbolic<PTI64>(P); break;
    }
    launch_sum_parts(st, P->list + P->bin_off[BIN_DENSE], P->bin_cnt[BIN_DENSE], P->nparts, P->part_count, P->nnz_col,
                     P->B.jc);
}

static spgemm_status_t finish_colptr(struct spgemm_plan* P) {
    spgemm_ctx* ctx = P->ctx;
    P->Ccp_buf = ctx_buf(ctx, 8 * (P->n + 1));
    if (!P->Ccp_buf) return set_err(ctx, SPGEMM_ERR_OOM, "colptr of C");
    P->Ccp = (int64_t*)P->Ccp_buf->p;
    {
        PhaseTimer t(ctx, SPGEMM_PHASE_SCAN, P->sr);
        launch_exclusive_scan(ctx->stream, P->nnz_col, P->n, P->Ccp, P->scan_tmp);
    }
    int64_t nnz = 0;
    SG_CUDA(ctx, cudaMemcpyAsync(&nnz, P->Ccp + P->n, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    SG_TRY(sync_ctx(ctx));
    P->nnzC = nnz;
    return SPGEMM_OK;
}

extern "C" {

spgemm_status_t spgemm_plan(spgemm_ctx_t ctx, spgemm_mat_t A, spgemm_mat_t B, spgemm_semiring_t sr,
                            const spgemm_opts_t* opts, spgemm_plan_t* out) {
    if (!ctx || !A || !B || !out) return SPGEMM_ERR_INVALID_ARG;
    SG_TRY(check_sr(ctx, sr));
    if (A->sr != sr || B->sr != sr) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "operand semiring differs from plan");
    if (A->n != B->m)
        return set_err(ctx, SPGEMM_ERR_DIM_MISMATCH, "A is %lld x %lld, B is %lld x %lld", (long long)A->m,
                       (long long)A->n, (long long)B->m, (long long)B->n);
    spgemm_opts_t o;
    spgemm_opts_default(&o);
    if (opts) o = *opts;
    auto* P = new struct spgemm_plan();
    DMat dA, dB;
    spgemm_status_t s = to_csc_operand(ctx, A, &P->Aconv, &dA);
    if (s == SPGEMM_OK) s = to_csc_operand(ctx, B, &P->Bconv, &dB);
    if (s == SPGEMM_OK) s = plan_build(ctx, dA, dB, sr, o, P);
    if (s != SPGEMM_OK) {
        spgemm_plan_destroy(P);
        return s;
    }
    *out = P;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_symbolic(spgemm_plan_t P, int64_t* nnz_C) {
    if (!P) return SPGEMM_ERR_INVALID_ARG;
    if (!P->symbolic_done) {
        run_symbolic_kernels(P);
        SG_CUDA(P->ctx, cudaGetLastError());
        SG_TRY(finish_colptr(P));
        P->symbolic_done = true;
    }
    if (nnz_C) *nnz_C = P->nnzC;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_numeric(spgemm_plan_t P, spgemm_mat_t* C) {
    if (!P || !C) return SPGEMM_ERR_INVALID_ARG;
    spgemm_ctx* ctx = P->ctx;
    if (!P->symbolic_done) SG_TRY(spgemm_symbolic(P, nullptr));
    const size_t w = sr_size(P->sr);
    auto rbuf = ctx_buf(ctx, 4 * (size_t)std::max<int64_t>(P->nnzC, 1));
    auto vbuf = ctx_buf(ctx, w * (size_t)std::max<int64_t>(P->nnzC, 1));
    if (!rbuf || !vbuf) return set_err(ctx, SPGEMM_ERR_OOM, "C arrays for nnz %lld", (long long)P->nnzC);
    switch (P->sr) {
    case SPGEMM_PLUS_TIMES_F64: dispatch_numeric<PT64>(P, (int32_t*)rbuf->p, vbuf->p); break;
    case SPGEMM_MIN_PLUS_F32: dispatch_numeric<MP32>(P, (int32_t*)rbuf->p, vbuf->p); break;
    case SPGEMM_OR_AND_BOOL: dispatch_numeric<BOOL8>(P, (int32_t*)rbuf->p, vbuf->p); break;
    case SPGEMM_PLUS_TIMES_I64: dispatch_numeric<PTI64>(P, (int32_t*)rbuf->p, vbuf->p); break;
    }
    SG_CUDA(ctx, cudaGetLastError());
    auto* M = new spgemm_mat();
    M->ctx = ctx;
    M->fmt = SPGEMM_FMT_CSC;
    M->sr = P->sr;
    M->m = P->m;
    M->n = P->n;
    M->nzc = P->n;
    M->nnz = P->nnzC;
    M->cp = P->Ccp;
    M->ir = (const int32_t*)rbuf->p;
    M->num = vbuf->p;
    M->owned = {P->Ccp_buf, rbuf, vbuf};
    *C = M;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_plan_stats(spgemm_plan_t P, int64_t* flops, int64_t* nnz_C, int64_t* tiers4,
                                  int64_t* overflow) {
    if (!P) return SPGEMM_ERR_INVALID_ARG;
    if (flops) *flops = P->flops_total;
    if (nnz_C) *nnz_C = P->nnzC;
    if (tiers4) {
        tiers4[0] = P->bin_cnt[0];
        tiers4[1] = 0;
        tiers4[2] = 0;
        for (int b = 1; b <= NWARP; ++b) tiers4[1] += P->bin_cnt[b];
        for (int b = NWARP + 1; b <= NWARP + NBLK; ++b) tiers4[2] += P->bin_cnt[b];
        tiers4[3] = P->bin_cnt[BIN_DENSE];
    }
    if (overflow) *overflow = P->overflow_cols;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_plan_tier_stats(spgemm_plan_t P, int64_t* cols4, int64_t* flops4, int64_t* nnz4,
                                       int64_t* bnnz4) {
    if (!P) return SPGEMM_ERR_INVALID_ARG;
    spgemm_ctx* ctx = P->ctx;
    auto buf = ctx_buf(ctx, 16 * 8);
    if (!buf) return set_err(ctx, SPGEMM_ERR_OOM, "tier stats");
    SG_CUDA(ctx, cudaMemsetAsync(buf->p, 0, 128, ctx->stream));
    launch_tier_stats(ctx->stream, P->bin, P->flops, P->nnz_col, P->B.jc, P->B.cp, P->B.nzc,
                      (unsigned long long*)buf->p);
    unsigned long long h[16];
    SG_CUDA(ctx, cudaMemcpyAsync(h, buf->p, 128, cudaMemcpyDeviceToHost, ctx->stream));
    SG_TRY(sync_ctx(ctx));
    for (int t = 0; t < 4; ++t) {
        if (cols4) cols4[t] = (int64_t)h[t];
        if (flops4) flops4[t] = (int64_t)h[4 + t];
        if (nnz4) nnz4[t] = P->symbolic_done ? (int64_t)h[8 + t] : -1;
        if (bnnz4) bnnz4[t] = (int64_t)h[12 + t];
    }
    return SPGEMM_OK;
}

spgemm_status_t spgemm_ctx_timing(spgemm_ctx_t ctx, int enable) {
    if (!ctx) return SPGEMM_ERR_INVALID_ARG;
    cudaStreamSynchronize(ctx->stream);
    for (auto& pe : ctx->pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    ctx->pending.clear();
    for (int i = 0; i < 4 * SPGEMM_NPHASE; ++i) {
        ctx->phase_ms[i] = 0;
        ctx->phase_cnt[i] = 0;
    }
    ctx->timing = enable != 0;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_ctx_phase_ms(spgemm_ctx_t ctx, double* ms, int64_t* count) {
    if (!ctx) return SPGEMM_ERR_INVALID_ARG;
    SG_TRY(sync_ctx(ctx));
    for (auto& pe : ctx->pending) {
        float t = 0;
        cudaEventElapsedTime(&t, pe.a, pe.b);
        ctx->phase_ms[pe.slot] += t;
        ctx->phase_cnt[pe.slot] += 1;
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    ctx->pending.clear();
    for (int i = 0; i < 4 * SPGEMM_NPHASE; ++i) {
        if (ms) ms[i] = ctx->phase_ms[i];
        if (count) count[i] = ctx->phase_cnt[i];
    }
    return SPGEMM_OK;
}

int64_t spgemm_launch_count(void) { return launches(); }

spgemm_status_t spgemm_plan_destroy(spgemm_plan_t P) {
    if (!P) return SPGEMM_ERR_INVALID_ARG;
    if (P->Aconv) spgemm_mat_destroy(P->Aconv);
    if (P->Bconv) spgemm_mat_destroy(P->Bconv);
    delete P;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_multiply(spgemm_ctx_t ctx, spgemm_mat_t A, spgemm_mat_t B, spgemm_semiring_t sr,
                                const spgemm_opts_t* opts, spgemm_mat_t* C) {
    spgemm_plan_t P = nullptr;
    SG_TRY(spgemm_plan(ctx, A, B, sr, opts, &P));
    spgemm_status_t s = spgemm_numeric(P, C);
    spgemm_plan_destroy(P);
    return s;
}

}  // extern "C"
