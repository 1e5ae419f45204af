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
        if (s != SPGEMM_OK) {
            // queued reads whose destinations the failing call is about to abandon
            ctx->rb_pending.clear();
            ctx->rb_used = 0;
        }
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
    const cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) {
        for (const auto& r : ctx->rb_pending) std::memcpy(r.dst, ctx->rb_host + r.off, r.bytes);
    }
    ctx->rb_pending.clear();
    ctx->rb_used = 0;
    SG_CUDA(ctx, e);
    SG_CUDA(ctx, cudaGetLastError());
    return SPGEMM_OK;
}

namespace {
// dst (mapped host memory) <- src (device), 8 bytes per thread when both are aligned
__global__ void k_read_back(unsigned char* __restrict__ dst, const unsigned char* __restrict__ src, size_t bytes) {
    const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, step = (size_t)gridDim.x * blockDim.x;
    if ((((uintptr_t)src | (uintptr_t)dst | bytes) & 7) == 0) {
        for (size_t i = i0; i < bytes / 8; i += step)
            reinterpret_cast<unsigned long long*>(dst)[i] = reinterpret_cast<const unsigned long long*>(src)[i];
    } else {
        for (size_t i = i0; i < bytes; i += step) dst[i] = src[i];
    }
}
}  // namespace

spgemm_status_t read_back(spgemm_ctx* ctx, void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return SPGEMM_OK;
    size_t off = (ctx->rb_used + 15) / 16 * 16;
    if (off + bytes > ctx->rb_cap) {
        if (!ctx->rb_pending.empty()) SG_TRY(sync_ctx(ctx));   // completes the queued reads first
        off = 0;
        if (bytes > ctx->rb_cap) {
            if (ctx->rb_host) {
                cudaStreamSynchronize(ctx->stream);   // no read still writes into the old buffer
                cudaFreeHost(ctx->rb_host);
            }
            ctx->rb_host = ctx->rb_dev = nullptr;
            ctx->rb_cap = 0;
            const size_t cap = std::max<size_t>((bytes + 4095) / 4096 * 4096, 64 * 1024);
            void* h = nullptr;
            SG_CUDA(ctx, cudaHostAlloc(&h, cap, cudaHostAllocMapped));
            void* d = nullptr;
            const cudaError_t e = cudaHostGetDevicePointer(&d, h, 0);
            if (e != cudaSuccess) {
                cudaFreeHost(h);
                return check_cuda(ctx, e, "mapped read-back buffer");
            }
            ctx->rb_host = (unsigned char*)h;
            ctx->rb_dev = (unsigned char*)d;
            ctx->rb_cap = cap;
        }
    }
    const int grid = (int)std::min<size_t>((bytes + 2047) / 2048, 256);
    k_read_back<<<grid, 256, 0, ctx->stream>>>(ctx->rb_dev + off, (const unsigned char*)src, bytes);
    note_launch();
    SG_CUDA(ctx, cudaGetLastError());
    ctx->rb_pending.push_back({dst, off, bytes});
    ctx->rb_used = off + bytes;
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
    o->block_max_flops = -1;
    o->dense_part_flops = DEFAULT_PART_FLOPS;
    o->range_slab_rows = 0;
    o->predictor_margin = 0.25f;
    o->check_inputs = 1;
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
    // a read left in flight by a failed call still writes the mapped buffer on the old stream
    if (ctx->rb_host && ctx->stream != (cudaStream_t)stream) cudaStreamSynchronize(ctx->stream);
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
    if (ctx->rb_host) cudaFreeHost(ctx->rb_host);
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

spgemm_plan::~spgemm_plan() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (Aconv) delete Aconv;
    if (Bconv) delete Bconv;
    for (auto* c : convs) delete c;
}

// ------------------------------------------------------------------ engine
DMat csc_view(int64_t m, int64_t n, int64_t nnz, const int64_t* cp, const int32_t* ir, const void* num) {
    DMat d;
    d.m = m;
    d.n = n;
    d.nzc = n;
    d.nnz = nnz;
    d.cp = cp;
    d.ir = ir;
    d.num = num;
    return d;
}

spgemm_mat_t new_owned_csc(spgemm_ctx* ctx, spgemm_semiring_t sr, int64_t m, int64_t n, int64_t nnz,
                           std::vector<std::shared_ptr<DevBuf>> owned, const int64_t* cp, const int32_t* ir,
                           const void* num) {
    auto* M = new spgemm_mat();
    M->ctx = ctx;
    M->fmt = SPGEMM_FMT_CSC;
    M->sr = sr;
    M->m = m;
    M->n = n;
    M->nzc = n;
    M->nnz = nnz;
    M->cp = cp;
    M->ir = ir;
    M->num = num;
    M->owned = std::move(owned);
    M->checked = true;
    return M;
}

spgemm_status_t to_csc_operand(spgemm_ctx* ctx, spgemm_mat_t M, spgemm_mat_t* conv, DMat* d) {
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

spgemm_status_t engine_setup(Engine* E, spgemm_ctx* ctx, spgemm_semiring_t sr, const spgemm_opts_t& opts,
                             std::vector<Prod> prods, bool want_features) {
    E->ctx = ctx;
    E->sr = sr;
    E->opts = opts;
    E->cfg.warp_max = std::max(0, std::min(opts.warp_max_flops, 512));
    int64_t mmax = 32;
    for (auto& pr : prods) mmax = std::max<int64_t>(mmax, pr.A.m);
    // automatic: operands of at most BLOCK_TIER_MAX_ROWS rows keep columns of up to 4096
    // flops in warp groups of the block tier; larger operands send columns beyond 1024
    // flops to the slab tier instead of the sorting CTA hash tables (measured best: R-MAT
    // 20 flat FP64 + bool 165.7 / 161.9 / 163.7 ms at 2048 / 1024 / 768)
    const int bm = opts.block_max_flops >= 0 ? opts.block_max_flops : (mmax <= BLOCK_TIER_MAX_ROWS ? 4096 : 1024);
    E->cfg.block_max = std::max(E->cfg.warp_max, std::min(bm, 4096));
    {
        // symbolic slabs: at most MAX_PARTS per column, each within the shared-memory bitmap
        const int64_t cap = opts.range_slab_rows > 0
                                ? std::min<int64_t>(std::max<int64_t>((opts.range_slab_rows + 31) / 32 * 32, 4096), 1 << 20)
                                : DEFAULT_SLAB_ROWS;
        const int64_t need = (ceil_div64(mmax, MAX_PARTS) + 32 + 31) / 32 * 32;
        E->cfg.dense_rows = (int)std::min<int64_t>({(mmax + 31) / 32 * 32, std::max(cap, need), int64_t(1) << 20});
        E->slab_rows_short = mmax > (int64_t)MAX_PARTS * (E->cfg.dense_rows - 32);
    }
    E->cfg.part_flops = std::max(1024, opts.dense_part_flops);
    cudaStream_t st = ctx->stream;
    {
        const cudaError_t pending = cudaGetLastError();
        if (pending != cudaSuccess)
            return set_err(ctx, SPGEMM_ERR_CUDA, "CUDA error pending before this call: %s", cudaGetErrorString(pending));
    }
    const int64_t np = (int64_t)prods.size();
    E->hitem_base.assign(np + 1, 0);
    int64_t bnz = 0, amax_n = 0;
    for (int64_t i = 0; i < np; ++i) {
        prods[i].item_base = E->hitem_base[i];
        prods[i].bnz_base = bnz;
        E->hitem_base[i + 1] = E->hitem_base[i] + prods[i].B.nzc;
        bnz += prods[i].B.nnz;
        amax_n += prods[i].A.n;
    }
    E->hprods = std::move(prods);
    const int64_t U = E->hitem_base[np];
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const int64_t U1 = std::max<int64_t>(U, 1);
    size_t o_prods = take(sizeof(Prod) * std::max<int64_t>(np, 1));
    size_t o_base = take(8 * (np + 1));
    size_t o_flops = take(8 * U1);
    size_t o_bin = take(U1);
    size_t o_iprod = take(4 * U1);
    size_t o_ctr = take(8 * (2 * NBIN + 8));
    size_t o_binoff = take(8 * NBIN);
    size_t o_list = take(sizeof(int2) * U1);
    size_t o_nnz = take(8 * U1);
    size_t o_scan = take(scan_tmp_bytes(U1));
    size_t o_nbin = take(U1);
    size_t o_nlist = take(sizeof(int2) * U1);
    size_t o_nctr = take(8 * 2 * NBIN);
    size_t o_nbinoff = take(8 * NBIN);
    size_t o_feat = want_features ? take(32 * U1) : 0;
    size_t o_sk = want_features ? take(8 * std::max<int64_t>(amax_n, 1)) : 0;
    size_t o_skb = want_features ? take(8 * (np + 1)) : 0;
    size_t o_mx = want_features ? take(8 * U1) : 0;
    // A-column cache for DCSC operands (SUMMA blocks): 12 bytes per entry of the B_i
    bool any_dcsc = false;
    for (auto& pr : E->hprods) any_dcsc = any_dcsc || pr.A.jc != nullptr;
    size_t o_acs = any_dcsc ? take(8 * std::max<int64_t>(bnz, 1)) : 0;
    size_t o_acl = any_dcsc ? take(4 * std::max<int64_t>(bnz, 1)) : 0;
    auto arena = ctx_buf(ctx, off);
    if (!arena) return set_err(ctx, SPGEMM_ERR_OOM, "engine arena of %zu bytes", off);
    E->bufs.push_back(arena);
    char* base = (char*)arena->p;
    Prod* dprods = (Prod*)(base + o_prods);
    int64_t* dbase = (int64_t*)(base + o_base);
    E->flops = (int64_t*)(base + o_flops);
    E->bin = (uint8_t*)(base + o_bin);
    E->item_prod = (int32_t*)(base + o_iprod);
    E->ctr = (unsigned long long*)(base + o_ctr);
    E->bin_off_dev = (int64_t*)(base + o_binoff);
    E->list = (int2*)(base + o_list);
    E->nnz_item = (int64_t*)(base + o_nnz);
    E->scan_tmp = base + o_scan;
    E->nbin = (uint8_t*)(base + o_nbin);
    E->nlist = (int2*)(base + o_nlist);
    E->nctr = (unsigned long long*)(base + o_nctr);
    E->nbin_off_dev = (int64_t*)(base + o_nbinoff);
    E->numeric_bins = false;
    SG_CUDA(ctx, cudaMemcpyAsync(dprods, E->hprods.data(), sizeof(Prod) * np, cudaMemcpyHostToDevice, st));
    SG_CUDA(ctx, cudaMemcpyAsync(dbase, E->hitem_base.data(), 8 * (np + 1), cudaMemcpyHostToDevice, st));
    E->it.prods = dprods;
    E->it.item_base = dbase;
    E->it.nprod = np;
    E->it.nitems = U;
    E->it.total_bnz = bnz;
    E->it.acs = any_dcsc ? (int64_t*)(base + o_acs) : nullptr;
    E->it.acl = any_dcsc ? (int32_t*)(base + o_acl) : nullptr;
    E->it.max_m = 0;
    for (auto& pr : E->hprods) E->it.max_m = std::max<int64_t>(E->it.max_m, pr.A.m);
    // operands of few rows: the sort tier takes the columns of 17 .. 128 products
    E->cfg.sort_max = E->it.max_m <= BLOCK_TIER_MAX_ROWS ? 128 : 0;
    uint64_t* sketch = nullptr;
    int64_t* skbase = nullptr;
    PhaseTimer t_an(ctx, SPGEMM_PHASE_ANALYZE, sr);
    if (want_features) {
        E->feat = (float*)(base + o_feat);
        E->maxlen = (int64_t*)(base + o_mx);
        sketch = (uint64_t*)(base + o_sk);
        skbase = (int64_t*)(base + o_skb);
        std::vector<int64_t> hb(np + 1, 0);
        for (int64_t i = 0; i < np; ++i) {
            hb[i + 1] = hb[i] + E->hprods[i].A.n;
            launch_row_sketch(st, E->hprods[i].A, sketch + hb[i]);
        }
        SG_CUDA(ctx, cudaMemcpyAsync(skbase, hb.data(), 8 * (np + 1), cudaMemcpyHostToDevice, st));
    }
    SG_CUDA(ctx, cudaMemsetAsync(E->ctr, 0, 8 * (2 * NBIN + 8), st));
    launch_analyze(st, E->it, E->cfg, E->flops, E->bin, E->item_prod, E->ctr, E->ctr + 2 * NBIN, sketch, skbase,
                   E->feat, E->maxlen);
    unsigned long long hc[NBIN + 1];
    SG_TRY(read_back(ctx, hc, E->ctr, sizeof(unsigned long long) * NBIN));
    SG_TRY(read_back(ctx, hc + NBIN, E->ctr + 2 * NBIN, sizeof(unsigned long long)));
    SG_TRY(sync_ctx(ctx));
    int64_t acc = 0;
    for (int b = 0; b < NBIN; ++b) {
        E->bin_cnt[b] = (int64_t)hc[b];
        E->bin_off[b] = acc;
        acc += E->bin_cnt[b];
    }
    E->flops_total = (int64_t)hc[NBIN];
    SG_CUDA(ctx, cudaMemcpyAsync(E->bin_off_dev, E->bin_off, sizeof(int64_t) * NBIN, cudaMemcpyHostToDevice, st));
    launch_bin_scatter(st, E->it, E->bin, E->item_prod, E->bin_off_dev, E->ctr + NBIN, E->list);
    const int64_t nd = E->bin_cnt[BIN_DENSE];
    E->dw = DenseWork();
    if (nd > 0 && E->it.max_m <= BLOCK_TIER_MAX_ROWS) {
        // operands of few rows: long columns are counted with row bitmaps and computed by the block tier
        DenseWork& dw = E->dw;
        dw.dlist = E->list + E->bin_off[BIN_DENSE];
        dw.ndense = nd;
        dw.dcol = true;
    } else if (nd > 0 && E->slab_rows_short)
        return set_err(ctx, SPGEMM_ERR_UNSUPPORTED,
                       "long columns of more than %d * (2^20 - 32) rows need more than %d row slabs", MAX_PARTS,
                       MAX_PARTS);
    if (nd > 0 && !E->dw.dcol) {
        // slabs of the long columns, then the slab arrays and row-set storage sized from them
        off = 0;
        size_t o_items = take(sizeof(int2) * nd * MAX_PARTS);
        size_t o_np = take(nd);
        size_t o_sb = take(4 * nd);
        size_t o_bb = take(8 * nd);
        auto dbuf = ctx_buf(ctx, off);
        if (!dbuf) return set_err(ctx, SPGEMM_ERR_OOM, "slab-tier arena of %zu bytes", off);
        E->bufs.push_back(dbuf);
        char* db = (char*)dbuf->p;
        DenseWork& dw = E->dw;
        dw.dlist = E->list + E->bin_off[BIN_DENSE];
        dw.ndense = nd;
        dw.items = (int2*)(db + o_items);
        dw.nitems = E->ctr + 2 * NBIN + 1;
        dw.nparts = (int8_t*)(db + o_np);
        dw.sbase = (int32_t*)(db + o_sb);
        dw.bbase = (int64_t*)(db + o_bb);
        unsigned long long* bnd_total = E->ctr + 2 * NBIN + 6;
        dw.store_ctr = E->ctr + 2 * NBIN + 2;
        dw.err = (int*)(E->ctr + 2 * NBIN + 3);
        unsigned long long* store_bound = E->ctr + 2 * NBIN + 4;
        dw.RB = E->cfg.dense_rows;
        launch_dense_items(st, E->it, dw.dlist, nd, E->flops, E->cfg.part_flops, dw.RB, (int2*)dw.items,
                           E->ctr + 2 * NBIN + 1, (int8_t*)dw.nparts, (int32_t*)dw.sbase, store_bound,
                           (int64_t*)dw.bbase, bnd_total);
        unsigned long long hs[3] = {0, 0, 0};
        SG_TRY(read_back(ctx, &hs[0], E->ctr + 2 * NBIN + 1, 8));
        SG_TRY(read_back(ctx, &hs[1], store_bound, 8));
        SG_TRY(read_back(ctx, &hs[2], bnd_total, 8));
        SG_TRY(sync_ctx(ctx));
        dw.nslabs = (int64_t)hs[0];
        dw.store_cap = (int64_t)hs[1];
        off = 0;
        const int64_t ns1 = std::max<int64_t>(dw.nslabs, 1);
        size_t o_cnt = take(4 * ns1);
        size_t o_pref = take(4 * ns1);
        size_t o_soff = take(8 * ns1);
        size_t o_rec = take(sizeof(SlabRec) * ns1);
        size_t o_store = take(4 * (size_t)std::max<int64_t>(dw.store_cap, 1));
        size_t o_bnd = take(4 * (size_t)std::max<unsigned long long>(hs[2], 1));
        auto sbuf = ctx_buf(ctx, off);
        if (!sbuf) return set_err(ctx, SPGEMM_ERR_OOM, "slab row sets of %zu bytes", off);
        E->bufs.push_back(sbuf);
        char* sb = (char*)sbuf->p;
        dw.scount = (int32_t*)(sb + o_cnt);
        dw.spref = (int32_t*)(sb + o_pref);
        dw.soff = (int64_t*)(sb + o_soff);
        dw.rec = (SlabRec*)(sb + o_rec);
        dw.store = (uint32_t*)(sb + o_store);
        dw.bnd = (int32_t*)(sb + o_bnd);
    }
    if (sr == SPGEMM_OR_AND_BOOL) {
        // boolean operands without a stored false value: the bitmap tiers take every output as true
        int* vals_zero = (int*)(E->ctr + 2 * NBIN + 5);
        if (ctx->bool_hint >= 0) SG_CUDA(ctx, cudaMemsetAsync(vals_zero, ctx->bool_hint ? 1 : 0, 4, st));
        else launch_false_values(st, E->it, vals_zero);
        E->dw.vals_zero = vals_zero;
    }
    SG_CUDA(ctx, cudaGetLastError());
    return SPGEMM_OK;
}

template <class SR>
static void dispatch_symbolic(Engine* E) {
    for (int which = 1; which <= 2; ++which) {
        PhaseTimer t(E->ctx, which == 1 ? SPGEMM_PHASE_SYMBOLIC_HASH : SPGEMM_PHASE_SYMBOLIC_DENSE, E->sr);
        launch_symbolic<SR>(E->ctx->stream, E->it, E->cfg, E->list, E->bin_off, E->bin_cnt, E->dw, E->nnz_item,
                            which);
    }
}

template <class SR>
static void dispatch_numeric(Engine* E, int32_t* Cir, void* Cv) {
    for (int which = 1; which <= 2; ++which) {
        PhaseTimer t(E->ctx, which == 1 ? SPGEMM_PHASE_NUMERIC_HASH : SPGEMM_PHASE_NUMERIC_DENSE, E->sr);
        const bool nb = which == 1 && E->numeric_bins;
        launch_numeric<SR>(E->ctx->stream, E->it, E->cfg, nb ? E->nlist : E->list, nb ? E->nbin_off : E->bin_off,
                           nb ? E->nbin_cnt : E->bin_cnt, E->dw, E->Coff, Cir, (typename SR::T*)Cv, which);
    }
}

spgemm_status_t engine_symbolic(Engine* E) {
    if (E->symbolic_done) return SPGEMM_OK;
    spgemm_ctx* ctx = E->ctx;
    cudaStream_t st = ctx->stream;
    const int64_t U = E->it.nitems;
    SG_CUDA(ctx, cudaMemsetAsync(E->nnz_item, 0, 8 * std::max<int64_t>(U, 1), st));
    switch (E->sr) {
    case SPGEMM_PLUS_TIMES_F64: dispatch_symbolic<PT64>(E); break;
    case SPGEMM_MIN_PLUS_F32: dispatch_symbolic<MP32>(E); break;
    case SPGEMM_OR_AND_BOOL: dispatch_symbolic<BOOL8>(E); break;
    case SPGEMM_PLUS_TIMES_I64: dispatch_symbolic<PTI64>(E); break;
    }
    SG_CUDA(ctx, cudaGetLastError());   // launch errors of the symbolic kernels
    launch_sum_parts(st, E->it, E->dw, E->nnz_item);
    E->Coff_buf = ctx_buf(ctx, 8 * (U + 1));
    if (!E->Coff_buf) return set_err(ctx, SPGEMM_ERR_OOM, "item offsets");
    E->Coff = (int64_t*)E->Coff_buf->p;
    {
        PhaseTimer t(ctx, SPGEMM_PHASE_SCAN, E->sr);
        launch_exclusive_scan(st, E->nnz_item, U, E->Coff, E->scan_tmp);
    }
    int64_t nnz = 0;
    int err = 0;
    unsigned long long nc[NBIN];
    {
        PhaseTimer t(ctx, SPGEMM_PHASE_SCAN, E->sr);
        SG_CUDA(ctx, cudaMemsetAsync(E->nctr, 0, 8 * 2 * NBIN, st));
        launch_numeric_bins(st, E->it, E->cfg, E->bin, E->flops, E->nnz_item, E->nbin, E->nctr);
    }
    SG_TRY(read_back(ctx, nc, E->nctr, sizeof(nc)));
    SG_TRY(read_back(ctx, &nnz, E->Coff + U, sizeof(int64_t)));
    SG_TRY(read_back(ctx, &err, E->ctr + 2 * NBIN + 3, sizeof(int)));
    // every product's first output, at the same synchronisation (batched calls)
    std::shared_ptr<DevBuf> pob;
    const int64_t np = E->it.nprod;
    if (E->want_prod_off && np > 1) {
        pob = ctx_buf(ctx, 8 * (np + 1));
        if (!pob) return set_err(ctx, SPGEMM_ERR_OOM, "product offsets");
        launch_gather_offsets(st, E->Coff, E->it.item_base, np, (int64_t*)pob->p);
        E->prod_off.assign(np + 1, 0);
        SG_TRY(read_back(ctx, E->prod_off.data(), pob->p, 8 * (np + 1)));
    }
    SG_TRY(sync_ctx(ctx));
    if (err) return set_err(ctx, SPGEMM_ERR_INDEX_OVERFLOW, "slab tier capacity exceeded (code %d)", err);
    E->nnz_total = nnz;
    if (E->want_prod_off && np <= 1) E->prod_off = {0, nnz};
    int64_t acc = 0;
    for (int b = 0; b < NBIN; ++b) {
        E->nbin_cnt[b] = (int64_t)nc[b];
        E->nbin_off[b] = acc;
        acc += E->nbin_cnt[b];
    }
    {
        PhaseTimer t(ctx, SPGEMM_PHASE_SCAN, E->sr);
        SG_CUDA(ctx, cudaMemcpyAsync(E->nbin_off_dev, E->nbin_off, sizeof(int64_t) * NBIN, cudaMemcpyHostToDevice, st));
        launch_bin_scatter(st, E->it, E->nbin, E->item_prod, E->nbin_off_dev, E->nctr + NBIN, E->nlist);
    }
    E->numeric_bins = true;
    E->symbolic_done = true;
    return SPGEMM_OK;
}

spgemm_status_t engine_alloc_out(Engine* E, std::shared_ptr<DevBuf>* rbuf, std::shared_ptr<DevBuf>* vbuf) {
    const size_t w = sr_size(E->sr);
    *rbuf = ctx_buf(E->ctx, 4 * (size_t)std::max<int64_t>(E->nnz_total, 1));
    *vbuf = ctx_buf(E->ctx, w * (size_t)std::max<int64_t>(E->nnz_total, 1));
    if (!*rbuf || !*vbuf) return set_err(E->ctx, SPGEMM_ERR_OOM, "output arrays for nnz %lld", (long long)E->nnz_total);
    return SPGEMM_OK;
}

spgemm_status_t engine_numeric(Engine* E, int32_t* Cir, void* Cv) {
    if (!E->symbolic_done) SG_TRY(engine_symbolic(E));
    switch (E->sr) {
    case SPGEMM_PLUS_TIMES_F64: dispatch_numeric<PT64>(E, Cir, Cv); break;
    case SPGEMM_MIN_PLUS_F32: dispatch_numeric<MP32>(E, Cir, Cv); break;
    case SPGEMM_OR_AND_BOOL: dispatch_numeric<BOOL8>(E, Cir, Cv); break;
    case SPGEMM_PLUS_TIMES_I64: dispatch_numeric<PTI64>(E, Cir, Cv); break;
    }
    SG_CUDA(E->ctx, cudaGetLastError());
    return SPGEMM_OK;
}

// C's column pointers for product 0 of E (n = B.n columns): the item offsets
// themselves when B is CSC, else a scatter over JC.
static spgemm_status_t product_colptr(Engine* E, std::shared_ptr<DevBuf>* cpbuf, const int64_t** cp) {
    const Prod& pr = E->hprods[0];
    if (pr.B.jc == nullptr && E->hprods.size() == 1) {
        *cpbuf = E->Coff_buf;
        *cp = E->Coff;
        return SPGEMM_OK;
    }
    const int64_t n = pr.B.n;
    auto buf = ctx_buf(E->ctx, 8 * (n + 1) + 16);
    if (!buf) return set_err(E->ctx, SPGEMM_ERR_OOM, "colptr");
    int64_t* cb = (int64_t*)buf->p;
    int64_t hb[2] = {0, n + 1};
    auto bb = ctx_buf(E->ctx, 16);
    if (!bb) return set_err(E->ctx, SPGEMM_ERR_OOM, "colptr base");
    SG_CUDA(E->ctx, cudaMemcpyAsync(bb->p, hb, 16, cudaMemcpyHostToDevice, E->ctx->stream));
    Items one = E->it;
    one.nprod = 1;
    launch_colptrs(E->ctx->stream, one, (const int64_t*)bb->p, n + 1, E->Coff, cb);
    SG_TRY(sync_ctx(E->ctx));   // keeps hb alive until the copy has run
    *cpbuf = buf;
    *cp = cb;
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
    if (o.check_inputs) SG_TRY(check_handles(ctx, {A, B}));
    auto* P = new struct spgemm_plan();
    P->ctx = ctx;
    P->sr = sr;
    P->opts = o;
    P->m = A->m;
    P->n = B->n;
    Prod pr;
    spgemm_status_t s = to_csc_operand(ctx, A, &P->Aconv, &pr.A);
    if (s == SPGEMM_OK) s = to_csc_operand(ctx, B, &P->Bconv, &pr.B);
    if (s == SPGEMM_OK) s = engine_setup(&P->E, ctx, sr, o, {pr}, o.use_predictor != 0);
    if (s != SPGEMM_OK) {
        spgemm_plan_destroy(P);
        return s;
    }
    *out = P;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_symbolic(spgemm_plan_t P, int64_t* nnz_C) {
    if (!P) return SPGEMM_ERR_INVALID_ARG;
    SG_TRY(engine_symbolic(&P->E));
    if (nnz_C) *nnz_C = P->E.nnz_total;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_numeric(spgemm_plan_t P, spgemm_mat_t* C) {
    if (!P || !C) return SPGEMM_ERR_INVALID_ARG;
    spgemm_ctx* ctx = P->ctx;
    Engine* E = &P->E;
    std::shared_ptr<DevBuf> rbuf, vbuf, cpbuf;
    if (P->opts.use_predictor && !E->symbolic_done) {
        // learned path: no symbolic pass for the hash tiers (predictor.cu)
        SG_TRY(engine_numeric_predicted(E, &rbuf, &vbuf));
    } else {
        SG_TRY(engine_symbolic(E));
        SG_TRY(engine_alloc_out(E, &rbuf, &vbuf));
        SG_TRY(engine_numeric(E, (int32_t*)rbuf->p, vbuf->p));
    }
    const int64_t* cp = nullptr;
    SG_TRY(product_colptr(E, &cpbuf, &cp));
    *C = new_owned_csc(ctx, P->sr, P->m, P->n, E->nnz_total, {cpbuf, rbuf, vbuf}, cp, (const int32_t*)rbuf->p,
                       vbuf->p);
    return SPGEMM_OK;
}

spgemm_status_t spgemm_plan_stats(spgemm_plan_t P, int64_t* flops, int64_t* nnz_C, int64_t* tiers4,
                                  int64_t* overflow) {
    if (!P) return SPGEMM_ERR_INVALID_ARG;
    const Engine& E = P->E;
    if (flops) *flops = E.flops_total;
    if (nnz_C) *nnz_C = E.nnz_total;
    if (tiers4) {
        tiers4[0] = E.bin_cnt[0];
        tiers4[1] = 0;
        tiers4[2] = 0;
        for (int b = BIN_TINY; b < BIN_BLK0; ++b) tiers4[1] += E.bin_cnt[b];
        for (int b = BIN_BLK0; b < BIN_DENSE; ++b) tiers4[2] += E.bin_cnt[b];
        tiers4[3] = E.bin_cnt[BIN_DENSE];
    }
    if (overflow) *overflow = E.overflow_items;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_plan_tier_stats(spgemm_plan_t P, int64_t* cols4, int64_t* flops4, int64_t* nnz4,
                                       int64_t* bnnz4) {
    if (!P) return SPGEMM_ERR_INVALID_ARG;
    spgemm_ctx* ctx = P->ctx;
    auto buf = ctx_buf(ctx, 16 * 8);
    if (!buf) return set_err(ctx, SPGEMM_ERR_OOM, "tier stats");
    SG_CUDA(ctx, cudaMemsetAsync(buf->p, 0, 128, ctx->stream));
    launch_tier_stats(ctx->stream, P->E.it, P->E.bin, P->E.item_prod, P->E.flops, P->E.nnz_item,
                      (unsigned long long*)buf->p);
    unsigned long long h[16];
    SG_TRY(read_back(ctx, h, buf->p, 128));
    SG_TRY(sync_ctx(ctx));
    for (int t = 0; t < 4; ++t) {
        if (cols4) cols4[t] = (int64_t)h[t];
        if (flops4) flops4[t] = (int64_t)h[4 + t];
        if (nnz4) nnz4[t] = P->E.symbolic_done ? (int64_t)h[8 + t] : -1;
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
    for (int i = 0; i < SPGEMM_NGROUP * 4 * SPGEMM_NPHASE; ++i) {
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
    for (int i = 0; i < SPGEMM_NGROUP * 4 * SPGEMM_NPHASE; ++i) {
        if (ms) ms[i] = ctx->phase_ms[i];
        if (count) count[i] = ctx->phase_cnt[i];
    }
    return SPGEMM_OK;
}

int64_t spgemm_launch_count(void) { return launches(); }

spgemm_status_t spgemm_ctx_timing_group(spgemm_ctx_t ctx, int group) {
    if (!ctx || group < 0 || group >= SPGEMM_NGROUP) return SPGEMM_ERR_INVALID_ARG;
    ctx->group = group;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_plan_destroy(spgemm_plan_t P) {
    if (!P) return SPGEMM_ERR_INVALID_ARG;
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
