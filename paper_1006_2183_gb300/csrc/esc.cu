// Expand-sort-compress (ESC) products: the data-parallel form of the
// hypersparse outer-product multiply of Section 2.4 (Fig. 10).
//
// The paper merges the outer products A(:,i) B(i,:), i in Isect, with a heap
// keyed by (column, row) and sums equal keys as they leave the heap.  Here every
// product of every item (product, column of B) is written out (expand), all of
// them are ordered by (item, row) with two stable radix passes (sort), and runs
// of equal keys are summed (compress).  Equal keys keep their expansion order,
// ascending k within a column, as in the heap merge.  No accumulator table is
// used, so the cost does not depend on the number of rows or on how a column's
// rows spread: the variant suits the most hypersparse block products, where the
// column tiers pay a per-column set-up for very little work.
#include <algorithm>

#include "internal.cuh"

using namespace sg;

namespace {

int grid_esc(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div64(n, 256), sm_count() * 32)); }

int bits_for(int64_t n) {
    int b = 0;
    while (b < 32 && (int64_t(1) << b) < n) ++b;
    return b;
}

// Expand: one warp per item writes the item's products at F[u] .. F[u+1) in
// (k, row) order: row keys, item ids and products.
template <class SR>
__global__ void k_esc_expand(Items it, const int32_t* __restrict__ item_prod, const int64_t* __restrict__ F,
                             int64_t u0, int64_t u1, uint32_t* __restrict__ krow, uint32_t* __restrict__ kitem,
                             typename SR::Acc* __restrict__ prod) {
    using T = typename SR::T;
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t f0 = __ldg(F + u0);
    for (int64_t u = u0 + wid; u < u1; u += nw) {
        if (__ldg(F + u + 1) == __ldg(F + u)) continue;
        const int pi = item_prod[u];
        const Prod* pr = it.prods + pi;
        const int64_t p = u - __ldg(it.item_base + pi);
        const int64_t bs = __ldg(pr->B.cp + p), be = __ldg(pr->B.cp + p + 1);
        int64_t out = __ldg(F + u) - f0;
        for (int64_t b0 = bs; b0 < be; b0 += 32) {
            const int64_t t = b0 + lane;
            int len = 0;
            int64_t a0 = 0;
            T bv = T(0);
            if (t < be) {
                int64_t s, en;
                a_col(it, pr, t, __ldg(pr->B.ir + t), s, en);
                a0 = s;
                len = (int)(en - s);
                bv = load_val<SR>(pr->B, t);
            }
            const int incl = warp_incl_scan(len);
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            for (int q0 = 0; q0 < total; q0 += 32) {
                const int q = q0 + lane;
                // owner lane j: the first with incl_j > q (5-step search over the shuffled prefix)
                int j = 0;
#pragma unroll
                for (int s = 16; s >= 1; s >>= 1) {
                    const int v = __shfl_sync(0xffffffffu, incl, j + s - 1);
                    if (v <= q) j += s;
                }
                j = j > 31 ? 31 : j;
                const int before = __shfl_sync(0xffffffffu, incl, j) - __shfl_sync(0xffffffffu, len, j);
                const int64_t aj = __shfl_sync(0xffffffffu, a0, j);
                const T bj = __shfl_sync(0xffffffffu, bv, j);
                if (q < total) {
                    const int64_t idx = aj + (q - before);
                    krow[out + q] = (uint32_t)__ldg(pr->A.ir + idx);
                    kitem[out + q] = (uint32_t)(u - u0);
                    prod[out + q] = SR::mul(load_val<SR>(pr->A, idx), bj);
                }
            }
            out += total;
        }
    }
}

__global__ void k_esc_iota(uint32_t* v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (uint32_t)i;
}

// second-pass keys: the item of each entry, in row-sorted order
__global__ void k_esc_item_keys(const uint32_t* __restrict__ idx, const uint32_t* __restrict__ kitem, int64_t n,
                                uint32_t* __restrict__ key) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        key[i] = kitem[idx[i]];
}

// run starts of equal (item, row) keys in the final order
__global__ void k_esc_flags(const uint32_t* __restrict__ idx, const uint32_t* __restrict__ item_sorted,
                            const uint32_t* __restrict__ krow, int64_t n, int64_t* __restrict__ flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = i == 0 || item_sorted[i] != item_sorted[i - 1] || krow[idx[i]] != krow[idx[i - 1]];
}

// compress: the first entry of every run sums the run (in expansion order) into its output slot
template <class SR>
__global__ void k_esc_compress(const uint32_t* __restrict__ idx, const uint32_t* __restrict__ krow,
                               const typename SR::Acc* __restrict__ prod, const int64_t* __restrict__ flag,
                               const int64_t* __restrict__ opos, int64_t n, int32_t* __restrict__ Cir,
                               typename SR::T* __restrict__ Cv) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const uint32_t e = idx[i];
        typename SR::Acc acc = prod[e];
        for (int64_t j = i + 1; j < n && !flag[j]; ++j) acc = SR::add(acc, prod[idx[j]]);
        const int64_t o = opos[i];
        Cir[o] = (int32_t)krow[e];
        Cv[o] = SR::out(acc);
    }
}

// item offsets of the chunk [u0, u1): the output position of the first entry of every
// item's segment (base = entries written by earlier chunks)
__global__ void k_esc_item_offsets(const int64_t* __restrict__ F, int64_t u0, int64_t u1,
                                   const int64_t* __restrict__ opos, int64_t n, int64_t base,
                                   int64_t* __restrict__ Coff) {
    const int64_t f0 = F[u0];
    for (int64_t u = u0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < u1; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = F[u] - f0;
        Coff[u] = base + (f < n ? opos[f] : opos[n]);
    }
}

// chunk boundaries: b[c] = first item u with F[u] >= c * lim (F ascending), b[nc] = U
__global__ void k_esc_bounds(const int64_t* __restrict__ F, int64_t U, int64_t lim, int64_t nc,
                             int64_t* __restrict__ b) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= nc; c += (int64_t)gridDim.x * blockDim.x) {
        if (c == nc) {
            b[c] = U;
            continue;
        }
        const int64_t v = c * lim;
        int64_t lo = 0, hi = U;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (F[mid] < v) lo = mid + 1;
            else hi = mid;
        }
        b[c] = lo;
    }
}

// Products per chunk: the work arrays take about 48 bytes per product.
constexpr int64_t ESC_CHUNK = int64_t(1) << 28;

template <class SR>
spgemm_status_t esc_run(Engine* E, std::shared_ptr<DevBuf>* rbuf_out, std::shared_ptr<DevBuf>* vbuf_out) {
    using Acc = typename SR::Acc;
    using T = typename SR::T;
    spgemm_ctx* ctx = E->ctx;
    cudaStream_t st = ctx->stream;
    const int64_t U = E->it.nitems;
    // expansion offsets
    auto Fb = ctx_buf(ctx, 8 * (U + 1) + scan_tmp_bytes(std::max<int64_t>(U, 1)));
    if (!Fb) return set_err(ctx, SPGEMM_ERR_OOM, "expansion offsets");
    int64_t* F = (int64_t*)Fb->p;
    launch_exclusive_scan(st, E->flops, U, F, F + (U + 1));
    int64_t Ttot = 0;
    SG_TRY(read_back(ctx, &Ttot, F + U, 8));
    SG_TRY(sync_ctx(ctx));
    // chunks of consecutive items holding about ESC_CHUNK products each
    const int64_t nc = std::max<int64_t>(1, ceil_div64(Ttot, ESC_CHUNK));
    std::vector<int64_t> hb(nc + 1), hf(nc + 1);
    {
        auto bb = ctx_buf(ctx, 8 * (nc + 1));
        if (!bb) return set_err(ctx, SPGEMM_ERR_OOM, "chunk bounds");
        k_esc_bounds<<<grid_esc(nc + 1), 256, 0, st>>>(F, U, ESC_CHUNK, nc, (int64_t*)bb->p);
        note_launch();
        SG_TRY(read_back(ctx, hb.data(), bb->p, 8 * (nc + 1)));
        SG_TRY(sync_ctx(ctx));
        for (int64_t c = 0; c <= nc; ++c)
            SG_TRY(read_back(ctx, &hf[c], F + hb[c], 8));
        SG_TRY(sync_ctx(ctx));
    }
    int64_t tmax = 1;
    for (int64_t c = 0; c < nc; ++c) tmax = std::max(tmax, hf[c + 1] - hf[c]);
    if (tmax >= (int64_t)UINT32_MAX)
        return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "expand-sort-compress: one column has %lld products", (long long)tmax);
    int64_t mmax = 1;
    for (auto& pr : E->hprods) mmax = std::max<int64_t>(mmax, pr.A.m);
    auto work = ctx_buf(ctx, 4 * 6 * tmax + sizeof(Acc) * tmax + 8 * (tmax + 1) * 2 + radix_tmp_bytes(tmax) +
                                 scan_tmp_bytes(tmax) + 4096);
    if (!work) return set_err(ctx, SPGEMM_ERR_OOM, "expand-sort-compress arrays for %lld products", (long long)tmax);
    char* w = (char*)work->p;
    auto take = [&](size_t bytes) {
        char* p = w;
        w += (bytes + 255) / 256 * 256;
        return p;
    };
    uint32_t* krow = (uint32_t*)take(4 * tmax);
    uint32_t* kitem = (uint32_t*)take(4 * tmax);
    uint32_t* k0 = (uint32_t*)take(4 * tmax);
    uint32_t* k1 = (uint32_t*)take(4 * tmax);
    uint32_t* v0 = (uint32_t*)take(4 * tmax);
    uint32_t* v1 = (uint32_t*)take(4 * tmax);
    Acc* prod = (Acc*)take(sizeof(Acc) * tmax);
    int64_t* flag = (int64_t*)take(8 * (tmax + 1));
    int64_t* opos = (int64_t*)take(8 * (tmax + 1));
    void* rtmp = take(radix_tmp_bytes(tmax));
    void* stmp = take(scan_tmp_bytes(tmax));
    E->Coff_buf = ctx_buf(ctx, 8 * (U + 1));
    if (!E->Coff_buf) return set_err(ctx, SPGEMM_ERR_OOM, "item offsets");
    E->Coff = (int64_t*)E->Coff_buf->p;
    std::vector<std::shared_ptr<DevBuf>> crb, cvb;
    std::vector<int64_t> cnnz;
    int64_t nnz = 0;
    for (int64_t c = 0; c < nc; ++c) {
        const int64_t u0 = hb[c], u1 = hb[c + 1], Tc = hf[c + 1] - hf[c];
        int64_t nc_nnz = 0;
        const uint32_t* idx = nullptr;
        if (Tc > 0) {
            k_esc_expand<SR><<<grid_esc((u1 - u0) * 32), 256, 0, st>>>(E->it, E->item_prod, F, u0, u1, krow, kitem,
                                                                       prod);
            k_esc_iota<<<grid_esc(Tc), 256, 0, st>>>(v0, Tc);
            note_launch(2);
            // (item, row) order by two stable LSD passes: rows, then items
            SG_CUDA(ctx, cudaMemcpyAsync(k0, krow, 4 * Tc, cudaMemcpyDeviceToDevice, st));
            bool second = false;
            radix_sort_pairs(st, k0, v0, k1, v1, Tc, bits_for(mmax), rtmp, &second);
            uint32_t* vr = second ? v1 : v0;    // entry ids in row order
            uint32_t* kA = second ? k0 : k1;    // free key buffer
            uint32_t* kB = second ? k1 : k0;    // the sorted rows, no longer needed
            uint32_t* vB = second ? v0 : v1;    // free value buffer
            k_esc_item_keys<<<grid_esc(Tc), 256, 0, st>>>(vr, kitem, Tc, kA);
            note_launch();
            bool second2 = false;
            radix_sort_pairs(st, kA, vr, kB, vB, Tc, bits_for(u1 - u0), rtmp, &second2);
            idx = second2 ? vB : vr;
            const uint32_t* items = second2 ? kB : kA;
            k_esc_flags<<<grid_esc(Tc), 256, 0, st>>>(idx, items, krow, Tc, flag);
            note_launch();
        }
        launch_exclusive_scan(st, flag, Tc, opos, stmp);
        SG_TRY(read_back(ctx, &nc_nnz, opos + Tc, 8));
        SG_TRY(sync_ctx(ctx));
        auto rb = ctx_buf(ctx, 4 * std::max<int64_t>(nc_nnz, 1));
        auto vb = ctx_buf(ctx, sizeof(T) * std::max<int64_t>(nc_nnz, 1));
        if (!rb || !vb) return set_err(ctx, SPGEMM_ERR_OOM, "expand-sort-compress output of %lld entries",
                                       (long long)nc_nnz);
        if (Tc > 0) {
            k_esc_compress<SR><<<grid_esc(Tc), 256, 0, st>>>(idx, krow, prod, flag, opos, Tc, (int32_t*)rb->p,
                                                              (T*)vb->p);
            note_launch();
        }
        if (u1 > u0) {
            k_esc_item_offsets<<<grid_esc(u1 - u0), 256, 0, st>>>(F, u0, u1, opos, Tc, nnz, E->Coff);
            note_launch();
        }
        crb.push_back(rb);
        cvb.push_back(vb);
        cnnz.push_back(nc_nnz);
        nnz += nc_nnz;
    }
    SG_CUDA(ctx, cudaMemcpyAsync(E->Coff + U, &nnz, 8, cudaMemcpyHostToDevice, st));
    std::shared_ptr<DevBuf> rb, vb;
    if (nc == 1) {
        rb = crb[0];
        vb = cvb[0];
    } else {
        rb = ctx_buf(ctx, 4 * std::max<int64_t>(nnz, 1));
        vb = ctx_buf(ctx, sizeof(T) * std::max<int64_t>(nnz, 1));
        if (!rb || !vb) return set_err(ctx, SPGEMM_ERR_OOM, "expand-sort-compress output of %lld entries", (long long)nnz);
        int64_t o = 0;
        for (size_t c = 0; c < crb.size(); ++c) {
            if (cnnz[c]) {
                SG_CUDA(ctx, cudaMemcpyAsync((int32_t*)rb->p + o, crb[c]->p, 4 * cnnz[c], cudaMemcpyDeviceToDevice, st));
                SG_CUDA(ctx, cudaMemcpyAsync((T*)vb->p + o, cvb[c]->p, sizeof(T) * cnnz[c], cudaMemcpyDeviceToDevice, st));
            }
            o += cnnz[c];
        }
    }
    SG_CUDA(ctx, cudaGetLastError());
    SG_TRY(sync_ctx(ctx));   // the work arrays and the host copy of nnz are released when this call returns
    E->nnz_total = nnz;
    E->symbolic_done = true;
    *rbuf_out = rb;
    *vbuf_out = vb;
    return SPGEMM_OK;
}

}  // namespace

spgemm_status_t engine_esc(Engine* E, std::shared_ptr<DevBuf>* rbuf, std::shared_ptr<DevBuf>* vbuf) {
    for (const Prod& pr : E->hprods)
        if (pr.row_base != 0 || pr.rb_cycle != 0)
            return set_err(E->ctx, SPGEMM_ERR_UNSUPPORTED, "expand-sort-compress writes local rows only");
    PhaseTimer t(E->ctx, SPGEMM_PHASE_NUMERIC_HASH, E->sr);
    switch (E->sr) {
    case SPGEMM_PLUS_TIMES_F64: return esc_run<PT64>(E, rbuf, vbuf);
    case SPGEMM_MIN_PLUS_F32: return esc_run<MP32>(E, rbuf, vbuf);
    case SPGEMM_OR_AND_BOOL: return esc_run<BOOL8>(E, rbuf, vbuf);
    case SPGEMM_PLUS_TIMES_I64: return esc_run<PTI64>(E, rbuf, vbuf);
    }
    return set_err(E->ctx, SPGEMM_ERR_INVALID_ARG, "bad semiring");
}
