// Numeric pass into upper-bound slots: no symbolic pass for the hash tiers.
//
// Every hash-tier column gets min(flops, m) output slots, an exact upper bound of
// its nnz, so the numeric kernels (in their counting mode) never overflow: they
// write the column at the start of its slots and record its exact count.  The
// range tier keeps its own symbolic pass (it also cuts the row ranges) and gets
// exact slots.  The result is a CSC with gaps, column u in
// [cap_off[u], cap_off[u] + nnz[u]), which a consumer that reads columns through
// (start, end) pairs takes as it is: the SUMMA stage merge reads its partial
// products this way, so the stage products skip the pass that only counts them.
#include <algorithm>

#include "internal.cuh"

using namespace sg;

namespace {

int gridb(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div64(n, 256), sm_count() * 8)); }

// slots per item: min(flops, m) for the hash tiers, the exact count for the range tier
__global__ void k_bound_capacity(Items it, const uint8_t* __restrict__ bin, const int32_t* __restrict__ item_prod,
                                 const int64_t* __restrict__ flops, const int64_t* __restrict__ nnz,
                                 int64_t* __restrict__ cap) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < it.nitems; u += (int64_t)gridDim.x * blockDim.x) {
        const int b = bin[u];
        if (b == BIN_DENSE) cap[u] = nnz[u];
        else if (b == 0) cap[u] = 0;
        else cap[u] = min(flops[u], it.prods[item_prod[u]].A.m);
    }
}

__global__ void k_col_ends(const int64_t* __restrict__ start, const int64_t* __restrict__ nnz, int64_t U,
                           int64_t* __restrict__ end) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < U; u += (int64_t)gridDim.x * blockDim.x)
        end[u] = start[u] + nnz[u];
}

template <class SR>
void numeric_launches(Engine* E, const int64_t* cap_off, int32_t* rows, void* vals) {
    cudaStream_t st = E->ctx->stream;
    {
        PhaseTimer t(E->ctx, SPGEMM_PHASE_NUMERIC_HASH, E->sr);
        launch_numeric_predicted<SR>(st, E->it, E->list, E->bin_off, E->bin_cnt, E->dw, cap_off, E->nnz_item, rows,
                                     (typename SR::T*)vals);
    }
    {
        PhaseTimer t(E->ctx, SPGEMM_PHASE_NUMERIC_DENSE, E->sr);
        launch_numeric<SR>(st, E->it, E->cfg, E->list, E->bin_off, E->bin_cnt, E->dw, cap_off, rows,
                           (typename SR::T*)vals, 2);
    }
}

template <class SR>
void range_symbolic(Engine* E) {
    launch_symbolic<SR>(E->ctx->stream, E->it, E->cfg, E->list, E->bin_off, E->bin_cnt, E->dw, E->nnz_item, 2);
}

}  // namespace

spgemm_status_t engine_numeric_bounded(Engine* E, std::shared_ptr<DevBuf>* rbuf, std::shared_ptr<DevBuf>* vbuf,
                                       std::shared_ptr<DevBuf>* colbuf, const int64_t** col_start,
                                       const int64_t** col_end) {
    spgemm_ctx* ctx = E->ctx;
    cudaStream_t st = ctx->stream;
    const int64_t U = E->it.nitems;
    const int64_t U1 = std::max<int64_t>(U, 1);
    const size_t w = sr_size(E->sr);
    SG_CUDA(ctx, cudaMemsetAsync(E->nnz_item, 0, 8 * U1, st));
    {
        PhaseTimer t(ctx, SPGEMM_PHASE_SYMBOLIC_DENSE, E->sr);
        switch (E->sr) {
        case SPGEMM_PLUS_TIMES_F64: range_symbolic<PT64>(E); break;
        case SPGEMM_MIN_PLUS_F32: range_symbolic<MP32>(E); break;
        case SPGEMM_OR_AND_BOOL: range_symbolic<BOOL8>(E); break;
        case SPGEMM_PLUS_TIMES_I64: range_symbolic<PTI64>(E); break;
        }
        launch_sum_parts(st, E->it, E->dw, E->nnz_item);
    }
    // slot offsets (U + 1) and column ends (U) in one buffer
    auto cb = ctx_buf(ctx, 8 * (2 * U1 + 2) + scan_tmp_bytes(U1));
    if (!cb) return set_err(ctx, SPGEMM_ERR_OOM, "slot offsets");
    int64_t* cap = (int64_t*)cb->p;                    // U: slots, then reused for the column ends
    int64_t* cap_off = cap + U1;                       // U + 1
    void* stmp = cap_off + (U1 + 1);
    int64_t total = 0;
    int err = 0;
    {
        PhaseTimer t(ctx, SPGEMM_PHASE_SCAN, E->sr);
        if (U > 0) {
            k_bound_capacity<<<gridb(U), 256, 0, st>>>(E->it, E->bin, E->item_prod, E->flops, E->nnz_item, cap);
            note_launch();
        }
        launch_exclusive_scan(st, cap, U, cap_off, stmp);
        SG_TRY(read_back(ctx, &total, cap_off + U, 8));
        SG_TRY(read_back(ctx, &err, E->ctr + 2 * NBIN + 3, sizeof(int)));
        SG_TRY(sync_ctx(ctx));
    }
    if (err) return set_err(ctx, SPGEMM_ERR_INDEX_OVERFLOW, "slab tier capacity exceeded (code %d)", err);
    auto r = ctx_buf(ctx, 4 * (size_t)std::max<int64_t>(total, 1));
    auto v = ctx_buf(ctx, w * (size_t)std::max<int64_t>(total, 1));
    if (!r || !v) return set_err(ctx, SPGEMM_ERR_OOM, "bounded output of %lld slots", (long long)total);
    switch (E->sr) {
    case SPGEMM_PLUS_TIMES_F64: numeric_launches<PT64>(E, cap_off, (int32_t*)r->p, v->p); break;
    case SPGEMM_MIN_PLUS_F32: numeric_launches<MP32>(E, cap_off, (int32_t*)r->p, v->p); break;
    case SPGEMM_OR_AND_BOOL: numeric_launches<BOOL8>(E, cap_off, (int32_t*)r->p, v->p); break;
    case SPGEMM_PLUS_TIMES_I64: numeric_launches<PTI64>(E, cap_off, (int32_t*)r->p, v->p); break;
    }
    if (U > 0) {
        k_col_ends<<<gridb(U), 256, 0, st>>>(cap_off, E->nnz_item, U, cap);
        note_launch();
    }
    // entries actually written (the statistics and the merge's nnz)
    int64_t nnz = 0;
    {
        auto sb = ctx_buf(ctx, 8 * (U1 + 1));
        if (!sb) return set_err(ctx, SPGEMM_ERR_OOM, "entry count");
        launch_exclusive_scan(st, E->nnz_item, U, (int64_t*)sb->p, stmp);
        SG_TRY(read_back(ctx, &nnz, (int64_t*)sb->p + U, 8));
        SG_TRY(sync_ctx(ctx));
    }
    SG_CUDA(ctx, cudaGetLastError());
    E->nnz_total = nnz;
    E->symbolic_done = true;
    *rbuf = r;
    *vbuf = v;
    *colbuf = cb;
    *col_start = cap_off;
    *col_end = cap;
    return SPGEMM_OK;
}
