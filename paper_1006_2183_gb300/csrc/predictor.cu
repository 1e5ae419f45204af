// Learned nnz(C(:,j)) predictor: a small MLP (8 -> 32 -> 32 -> 1, ReLU, fp32)
// over per-column features, trained and evaluated by the kernels below.  The
// paper has no predictor; its Section 8 names structure prediction as future
// work.  The product uses it to size the output without the symbolic pass;
// every column still gets its exact count from the numeric pass, and columns
// whose count exceeds the predicted capacity are recomputed into their exact
// place, so the result does not depend on the prediction.
//
// Parameter layout (row-major W[out][in]):
//   W1[32][8], b1[32], W2[32][32], b2[32], w3[32], b3   (1377 floats)
// Inputs per column (written by k_analyze):
//   log1p d, log1p flops, log1p max len, log1p m, log1p lc, log1p min(flops, m),
//   log1p(flops - max len), popcount(sketch) / 64
// with d = nnz(B(:,j)), len = nnz(A(:,k)) over k in B(:,j), sketch = OR of
// per-column 64-bit row sketches (bit = bits 31..26 of row * 0x9E3779B1) and
// lc = 64 ln(64 / (64 - min(popcount, 63.5))) (linear counting).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

using namespace sg;

namespace {

constexpr int NP = SPGEMM_PREDICTOR_NPARAM;
constexpr int O_W1 = 0, O_B1 = 256, O_W2 = 288, O_B2 = 1312, O_W3 = 1344, O_B3 = 1376;

__device__ __forceinline__ float mlp_eval(const float* __restrict__ th, const float* x, float* z1, float* z2) {
    float h1[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        float a = th[O_B1 + i];
#pragma unroll
        for (int f = 0; f < 8; ++f) a = fmaf(th[O_W1 + i * 8 + f], x[f], a);
        if (z1) z1[i] = a;
        h1[i] = a > 0.f ? a : 0.f;
    }
    float y = th[O_B3];
#pragma unroll 4
    for (int j = 0; j < 32; ++j) {
        float a = th[O_B2 + j];
#pragma unroll
        for (int i = 0; i < 32; ++i) a = fmaf(th[O_W2 + j * 32 + i], h1[i], a);
        if (z2) z2[j] = a;
        y = fmaf(th[O_W3 + j], a > 0.f ? a : 0.f, y);
    }
    return y;
}

__global__ void __launch_bounds__(256) k_mlp_forward(const float* __restrict__ theta, const float* __restrict__ X,
                                                     int64_t N, float* __restrict__ out) {
    __shared__ float th[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) th[i] = theta[i];
    __syncthreads();
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        float x[8];
#pragma unroll
        for (int f = 0; f < 8; ++f) x[f] = X[s * 8 + f];
        out[s] = mlp_eval(th, x, nullptr, nullptr);
    }
}

// Per-sample backpropagation of L = (1/N) sum (y - t)^2; contributions are
// summed over the warp with shuffles, then into shared memory, then globally.
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ theta, const float* __restrict__ X,
                                                  const float* __restrict__ T, int64_t N, float* __restrict__ grad,
                                                  float* __restrict__ loss) {
    __shared__ float th[NP];
    __shared__ float g[NP];
    __shared__ float s_loss;
    for (int i = threadIdx.x; i < NP; i += blockDim.x) {
        th[i] = theta[i];
        g[i] = 0.f;
    }
    if (threadIdx.x == 0) s_loss = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const float invN = 1.0f / (float)N;
    for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x; s0 < N; s0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = s0 + threadIdx.x;
        const bool ok = s < N;
        float x[8], z1[32], z2[32];
#pragma unroll
        for (int f = 0; f < 8; ++f) x[f] = ok ? X[s * 8 + f] : 0.f;
        const float y = mlp_eval(th, x, z1, z2);
        const float dy = ok ? 2.0f * (y - T[s]) * invN : 0.f;
        const float l = ok ? (y - T[s]) * (y - T[s]) * invN : 0.f;
        auto wsum = [&](float v) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            return v;
        };
        float ls = wsum(l);
        if (lane == 0) atomicAdd(&s_loss, ls);
        float gb3 = wsum(dy);
        if (lane == 0) atomicAdd(&g[O_B3], gb3);
        float dz2[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float h2 = z2[j] > 0.f ? z2[j] : 0.f;
            float v = wsum(dy * h2);
            if (lane == 0) atomicAdd(&g[O_W3 + j], v);
            dz2[j] = z2[j] > 0.f ? dy * th[O_W3 + j] : 0.f;
            v = wsum(dz2[j]);
            if (lane == 0) atomicAdd(&g[O_B2 + j], v);
        }
        float h1[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) h1[i] = z1[i] > 0.f ? z1[i] : 0.f;
        for (int j = 0; j < 32; ++j) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                float v = wsum(dz2[j] * h1[i]);
                if (lane == 0) atomicAdd(&g[O_W2 + j * 32 + i], v);
            }
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            float dh = 0.f;
#pragma unroll
            for (int j = 0; j < 32; ++j) dh = fmaf(dz2[j], th[O_W2 + j * 32 + i], dh);
            const float dz1 = z1[i] > 0.f ? dh : 0.f;
            float v = wsum(dz1);
            if (lane == 0) atomicAdd(&g[O_B1 + i], v);
#pragma unroll
            for (int f = 0; f < 8; ++f) {
                float w = wsum(dz1 * x[f]);
                if (lane == 0) atomicAdd(&g[O_W1 + i * 8 + f], w);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NP; i += blockDim.x)
        if (g[i] != 0.f) atomicAdd(grad + i, g[i]);
    if (threadIdx.x == 0) atomicAdd(loss, s_loss);
}

// Adam (Kingma & Ba 2015) with bias correction.
__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, int t, float lr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NP) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)t));
    const float vh = vi / (1.f - powf(b2, (float)t));
    theta[i] -= lr * mh / (sqrtf(vh) + eps);
}

// Output capacity per item from the prediction: ceil((1 + margin) * expm1(y)) + 2,
// clamped to the exact bounds [max_k nnz(A(:,k)), min(flops, m)].  Items of the
// range tier keep their exact count (already in cap).
__global__ void __launch_bounds__(256) k_mlp_capacity(const float* __restrict__ theta, Items it,
                                                      const float* __restrict__ feat, const uint8_t* __restrict__ bin,
                                                      const int32_t* __restrict__ item_prod,
                                                      const int64_t* __restrict__ flops,
                                                      const int64_t* __restrict__ maxlen, float margin,
                                                      int64_t* __restrict__ cap) {
    __shared__ float th[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) th[i] = theta[i];
    __syncthreads();
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < it.nitems;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int b = bin[u];
        if (b == 0) {
            cap[u] = 0;
            continue;
        }
        if (b == BIN_DENSE) continue;
        float x[8];
#pragma unroll
        for (int f = 0; f < 8; ++f) x[f] = feat[u * 8 + f];
        const float y = mlp_eval(th, x, nullptr, nullptr);
        const float pred = expm1f(fminf(y, 40.f));
        const int64_t m = it.prods[item_prod[u]].A.m;
        const int64_t hi = flops[u] < m ? flops[u] : m;
        const int64_t lo = maxlen[u];
        double c = ceil((1.0 + (double)margin) * (double)fmaxf(pred, 0.f)) + 2.0;
        int64_t ci = c > (double)hi ? hi : (int64_t)c;
        cap[u] = ci < lo ? lo : ci;
    }
}

// Items of the hash tiers whose count exceeded their capacity, re-binned by flops.
__global__ void k_overflow_lists(Items it, const int2* __restrict__ list, int64_t n, const uint8_t* __restrict__ bin,
                                 const int64_t* __restrict__ nnz, const int64_t* __restrict__ cap_off,
                                 const int64_t* __restrict__ bin_off, unsigned long long* __restrict__ cursor,
                                 int2* __restrict__ olist) {
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n; w += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = list[w];
        const int64_t u = it.item_base[e.x] + e.y;
        const int64_t cp = cap_off[u + 1] - cap_off[u];
        if (nnz[u] > cp) {
            const int b = bin[u];
            const unsigned long long q = atomicAdd(cursor + b, 1ull);
            olist[bin_off[b] + q] = e;
        }
    }
}

// Move every item that fitted from the predicted layout to its exact place (warp per item).
template <int W>
__global__ void k_move_items(int64_t U, const int64_t* __restrict__ nnz, const int64_t* __restrict__ cap_off,
                             const int64_t* __restrict__ exact_off, const int32_t* __restrict__ tir,
                             const void* __restrict__ tv, int32_t* __restrict__ ir, void* __restrict__ v) {
    using Wt = typename std::conditional<W == 1, uint8_t, typename std::conditional<W == 4, uint32_t, uint64_t>::type>::type;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < U; u += warps) {
        const int64_t c = nnz[u];
        const int64_t s = cap_off[u];
        if (c > cap_off[u + 1] - s) continue;   // overflowed: recomputed in place later
        const int64_t d = exact_off[u];
        for (int64_t i = lane; i < c; i += 32) {
            ir[d + i] = tir[s + i];
            reinterpret_cast<Wt*>(v)[d + i] = reinterpret_cast<const Wt*>(tv)[s + i];
        }
    }
}

spgemm_status_t ensure_pred(spgemm_ctx* ctx) {
    if (ctx->pred) return SPGEMM_OK;
    ctx->pred = (float*)ctx_alloc(ctx, 4 * NP);
    ctx->adam_m = (float*)ctx_alloc(ctx, 4 * NP);
    ctx->adam_v = (float*)ctx_alloc(ctx, 4 * NP);
    ctx->grad = (float*)ctx_alloc(ctx, 4 * (NP + 1));
    if (!ctx->pred || !ctx->adam_m || !ctx->adam_v || !ctx->grad) return set_err(ctx, SPGEMM_ERR_OOM, "predictor state");
    SG_CUDA(ctx, cudaMemsetAsync(ctx->adam_m, 0, 4 * NP, ctx->stream));
    SG_CUDA(ctx, cudaMemsetAsync(ctx->adam_v, 0, 4 * NP, ctx->stream));
    return SPGEMM_OK;
}

int gridp(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div64(n, 256), sm_count() * 8)); }

}  // namespace

// The predicted execution of an engine (see api.cu for the exact one).
spgemm_status_t engine_numeric_predicted(Engine* E, std::shared_ptr<DevBuf>* rbuf_out, std::shared_ptr<DevBuf>* vbuf_out) {
    spgemm_ctx* ctx = E->ctx;
    cudaStream_t st = ctx->stream;
    if (!ctx->pred_ready) return set_err(ctx, SPGEMM_ERR_STATE, "predictor parameters are not set");
    if (!E->feat || !E->maxlen) return set_err(ctx, SPGEMM_ERR_STATE, "engine was set up without features");
    const int64_t U = E->it.nitems;
    const size_t w = sr_size(E->sr);
    // exact counts for the range tier come from its own symbolic pass (it also cuts the ranges)
    SG_CUDA(ctx, cudaMemsetAsync(E->nnz_item, 0, 8 * std::max<int64_t>(U, 1), st));
    {
        PhaseTimer t(ctx, SPGEMM_PHASE_SYMBOLIC_DENSE, E->sr);
        switch (E->sr) {
        case SPGEMM_PLUS_TIMES_F64: launch_symbolic<PT64>(st, E->it, E->cfg, E->list, E->bin_off, E->bin_cnt, E->dw, E->nnz_item, 2); break;
        case SPGEMM_MIN_PLUS_F32: launch_symbolic<MP32>(st, E->it, E->cfg, E->list, E->bin_off, E->bin_cnt, E->dw, E->nnz_item, 2); break;
        case SPGEMM_OR_AND_BOOL: launch_symbolic<BOOL8>(st, E->it, E->cfg, E->list, E->bin_off, E->bin_cnt, E->dw, E->nnz_item, 2); break;
        case SPGEMM_PLUS_TIMES_I64: launch_symbolic<PTI64>(st, E->it, E->cfg, E->list, E->bin_off, E->bin_cnt, E->dw, E->nnz_item, 2); break;
        }
        launch_sum_parts(st, E->it, E->dw, E->nnz_item);
    }
    // capacities: predicted for the hash tiers, exact for the range tier, 0 for empty columns
    auto capb = ctx_buf(ctx, 8 * (2 * (U + 1)) + 8 * (2 * NBIN + 2));
    if (!capb) return set_err(ctx, SPGEMM_ERR_OOM, "capacities");
    int64_t* cap = (int64_t*)capb->p;
    int64_t* cap_off = cap + (U + 1);
    unsigned long long* octr = (unsigned long long*)(cap_off + (U + 1));
    int64_t total_cap = 0;
    {
        PhaseTimer t(ctx, SPGEMM_PHASE_PREDICT, E->sr);
        SG_CUDA(ctx, cudaMemcpyAsync(cap, E->nnz_item, 8 * std::max<int64_t>(U, 1), cudaMemcpyDeviceToDevice, st));
        if (U > 0) {
            k_mlp_capacity<<<gridp(U), 256, 0, st>>>(ctx->pred, E->it, E->feat, E->bin, E->item_prod, E->flops,
                                                     E->maxlen, E->opts.predictor_margin, cap);
            note_launch();
        }
        launch_exclusive_scan(st, cap, U, cap_off, E->scan_tmp);
        SG_TRY(read_back(ctx, &total_cap, cap_off + U, 8));
        SG_TRY(sync_ctx(ctx));
    }
    auto trb = ctx_buf(ctx, 4 * (size_t)std::max<int64_t>(total_cap, 1));
    auto tvb = ctx_buf(ctx, w * (size_t)std::max<int64_t>(total_cap, 1));
    if (!trb || !tvb) return set_err(ctx, SPGEMM_ERR_OOM, "predicted output of %lld entries", (long long)total_cap);
    // numeric into the predicted layout; hash tiers record their exact counts
    {
        PhaseTimer t(ctx, SPGEMM_PHASE_NUMERIC_HASH, E->sr);
        switch (E->sr) {
        case SPGEMM_PLUS_TIMES_F64: launch_numeric_predicted<PT64>(st, E->it, E->list, E->bin_off, E->bin_cnt, E->dw, cap_off, E->nnz_item, (int32_t*)trb->p, (double*)tvb->p); break;
        case SPGEMM_MIN_PLUS_F32: launch_numeric_predicted<MP32>(st, E->it, E->list, E->bin_off, E->bin_cnt, E->dw, cap_off, E->nnz_item, (int32_t*)trb->p, (float*)tvb->p); break;
        case SPGEMM_OR_AND_BOOL: launch_numeric_predicted<BOOL8>(st, E->it, E->list, E->bin_off, E->bin_cnt, E->dw, cap_off, E->nnz_item, (int32_t*)trb->p, (uint8_t*)tvb->p); break;
        case SPGEMM_PLUS_TIMES_I64: launch_numeric_predicted<PTI64>(st, E->it, E->list, E->bin_off, E->bin_cnt, E->dw, cap_off, E->nnz_item, (int32_t*)trb->p, (int64_t*)tvb->p); break;
        }
    }
    {
        PhaseTimer t(ctx, SPGEMM_PHASE_NUMERIC_DENSE, E->sr);
        switch (E->sr) {
        case SPGEMM_PLUS_TIMES_F64: launch_numeric<PT64>(st, E->it, E->cfg, E->list, E->bin_off, E->bin_cnt, E->dw, cap_off, (int32_t*)trb->p, (double*)tvb->p, 2); break;
        case SPGEMM_MIN_PLUS_F32: launch_numeric<MP32>(st, E->it, E->cfg, E->list, E->bin_off, E->bin_cnt, E->dw, cap_off, (int32_t*)trb->p, (float*)tvb->p, 2); break;
        case SPGEMM_OR_AND_BOOL: launch_numeric<BOOL8>(st, E->it, E->cfg, E->list, E->bin_off, E->bin_cnt, E->dw, cap_off, (int32_t*)trb->p, (uint8_t*)tvb->p, 2); break;
        case SPGEMM_PLUS_TIMES_I64: launch_numeric<PTI64>(st, E->it, E->cfg, E->list, E->bin_off, E->bin_cnt, E->dw, cap_off, (int32_t*)trb->p, (int64_t*)tvb->p, 2); break;
        }
    }
    // exact offsets, overflowed items
    E->Coff_buf = ctx_buf(ctx, 8 * (U + 1));
    auto olb = ctx_buf(ctx, sizeof(int2) * std::max<int64_t>(E->bin_off[BIN_DENSE], 1));
    if (!E->Coff_buf || !olb) return set_err(ctx, SPGEMM_ERR_OOM, "exact offsets");
    E->Coff = (int64_t*)E->Coff_buf->p;
    int2* olist = (int2*)olb->p;
    int64_t nnz = 0;
    unsigned long long ocnt[NBIN];
    {
        PhaseTimer t(ctx, SPGEMM_PHASE_PREDICT, E->sr);
        launch_exclusive_scan(st, E->nnz_item, U, E->Coff, E->scan_tmp);
        SG_CUDA(ctx, cudaMemsetAsync(octr, 0, 8 * NBIN, st));
        const int64_t nh = E->bin_off[BIN_DENSE] - E->bin_off[1];
        if (nh > 0) {
            k_overflow_lists<<<gridp(nh), 256, 0, st>>>(E->it, E->list + E->bin_off[1], nh, E->bin, E->nnz_item, cap_off,
                                                        E->bin_off_dev, octr, olist);
            note_launch();
        }
        SG_TRY(read_back(ctx, &nnz, E->Coff + U, 8));
        SG_TRY(read_back(ctx, ocnt, octr, 8 * NBIN));
        SG_TRY(sync_ctx(ctx));
    }
    E->nnz_total = nnz;
    E->symbolic_done = true;
    E->overflow_items = 0;
    int64_t ocnt64[NBIN];
    for (int b = 0; b < NBIN; ++b) {
        ocnt64[b] = (int64_t)ocnt[b];
        if (b > 0 && b < BIN_DENSE) E->overflow_items += ocnt64[b];
    }
    std::shared_ptr<DevBuf> rbuf, vbuf;
    SG_TRY(engine_alloc_out(E, &rbuf, &vbuf));
    {
        PhaseTimer t(ctx, SPGEMM_PHASE_PREDICT, E->sr);
        if (U > 0) {
            const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div64(U * 32, 256), sm_count() * 16));
            switch (w) {
            case 1: k_move_items<1><<<grid, 256, 0, st>>>(U, E->nnz_item, cap_off, E->Coff, (int32_t*)trb->p, tvb->p, (int32_t*)rbuf->p, vbuf->p); break;
            case 4: k_move_items<4><<<grid, 256, 0, st>>>(U, E->nnz_item, cap_off, E->Coff, (int32_t*)trb->p, tvb->p, (int32_t*)rbuf->p, vbuf->p); break;
            default: k_move_items<8><<<grid, 256, 0, st>>>(U, E->nnz_item, cap_off, E->Coff, (int32_t*)trb->p, tvb->p, (int32_t*)rbuf->p, vbuf->p); break;
            }
            note_launch();
        }
        if (E->overflow_items > 0) {
            // overflowed columns: exact numeric pass straight into their final place
            switch (E->sr) {
            case SPGEMM_PLUS_TIMES_F64: launch_numeric<PT64>(st, E->it, E->cfg, olist, E->bin_off, ocnt64, E->dw, E->Coff, (int32_t*)rbuf->p, (double*)vbuf->p, 1); break;
            case SPGEMM_MIN_PLUS_F32: launch_numeric<MP32>(st, E->it, E->cfg, olist, E->bin_off, ocnt64, E->dw, E->Coff, (int32_t*)rbuf->p, (float*)vbuf->p, 1); break;
            case SPGEMM_OR_AND_BOOL: launch_numeric<BOOL8>(st, E->it, E->cfg, olist, E->bin_off, ocnt64, E->dw, E->Coff, (int32_t*)rbuf->p, (uint8_t*)vbuf->p, 1); break;
            case SPGEMM_PLUS_TIMES_I64: launch_numeric<PTI64>(st, E->it, E->cfg, olist, E->bin_off, ocnt64, E->dw, E->Coff, (int32_t*)rbuf->p, (int64_t*)vbuf->p, 1); break;
            }
        }
    }
    SG_CUDA(ctx, cudaGetLastError());
    // the temporaries are released in stream order after the kernels above
    *rbuf_out = rbuf;
    *vbuf_out = vbuf;
    return SPGEMM_OK;
}

extern "C" {

spgemm_status_t spgemm_predictor_set(spgemm_ctx_t ctx, const float* params) {
    if (!ctx || !params) return SPGEMM_ERR_INVALID_ARG;
    SG_TRY(ensure_pred(ctx));
    SG_CUDA(ctx, cudaMemcpyAsync(ctx->pred, params, 4 * NP, cudaMemcpyHostToDevice, ctx->stream));
    SG_CUDA(ctx, cudaMemsetAsync(ctx->adam_m, 0, 4 * NP, ctx->stream));
    SG_CUDA(ctx, cudaMemsetAsync(ctx->adam_v, 0, 4 * NP, ctx->stream));
    SG_TRY(sync_ctx(ctx));
    ctx->adam_t = 0;
    ctx->pred_ready = true;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_predictor_get(spgemm_ctx_t ctx, float* params) {
    if (!ctx || !params) return SPGEMM_ERR_INVALID_ARG;
    if (!ctx->pred_ready) return set_err(ctx, SPGEMM_ERR_STATE, "predictor parameters are not set");
    SG_TRY(read_back(ctx, params, ctx->pred, 4 * NP));
    return sync_ctx(ctx);
}

spgemm_status_t spgemm_predictor_features(spgemm_ctx_t ctx, spgemm_mat_t A, spgemm_mat_t B, float* X, int64_t* nnz) {
    if (!ctx || !A || !B || !X) return SPGEMM_ERR_INVALID_ARG;
    if (A->n != B->m) return set_err(ctx, SPGEMM_ERR_DIM_MISMATCH, "inner dimensions differ");
    if (B->fmt != SPGEMM_FMT_CSC || A->fmt == SPGEMM_FMT_CSR)
        return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "features need CSC or DCSC A and CSC B");
    SG_TRY(check_handles(ctx, {A, B}));
    spgemm_opts_t o;
    spgemm_opts_default(&o);
    Prod pr;
    pr.A = dmat_of(A);
    pr.B = dmat_of(B);
    Engine E;
    SG_TRY(engine_setup(&E, ctx, A->sr, o, {pr}, true));
    SG_CUDA(ctx, cudaMemcpyAsync(X, E.feat, 32 * (size_t)B->n, cudaMemcpyDeviceToDevice, ctx->stream));
    if (nnz) {
        SG_TRY(engine_symbolic(&E));
        SG_CUDA(ctx, cudaMemcpyAsync(nnz, E.nnz_item, 8 * (size_t)B->n, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return sync_ctx(ctx);
}

spgemm_status_t spgemm_predictor_train_step(spgemm_ctx_t ctx, const float* X, const float* y, int64_t N, float lr,
                                            float* loss_host, float* grad_host) {
    if (!ctx || !X || !y || N <= 0) return SPGEMM_ERR_INVALID_ARG;
    if (!ctx->pred_ready) return set_err(ctx, SPGEMM_ERR_STATE, "predictor parameters are not set");
    cudaStream_t st = ctx->stream;
    SG_CUDA(ctx, cudaMemsetAsync(ctx->grad, 0, 4 * (NP + 1), st));
    k_mlp_grad<<<gridp(N), 256, 0, st>>>(ctx->pred, X, y, N, ctx->grad, ctx->grad + NP);
    note_launch();
    if (grad_host) SG_TRY(read_back(ctx, grad_host, ctx->grad, 4 * NP));
    float l = 0.f;
    SG_TRY(read_back(ctx, &l, ctx->grad + NP, 4));
    ctx->adam_t += 1;
    k_adam<<<(NP + 255) / 256, 256, 0, st>>>(ctx->pred, ctx->grad, ctx->adam_m, ctx->adam_v, ctx->adam_t, lr);
    note_launch();
    SG_TRY(sync_ctx(ctx));
    if (loss_host) *loss_host = l;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_predictor_forward(spgemm_ctx_t ctx, const float* X, int64_t N, float* pred) {
    if (!ctx || !X || !pred || N < 0) return SPGEMM_ERR_INVALID_ARG;
    if (!ctx->pred_ready) return set_err(ctx, SPGEMM_ERR_STATE, "predictor parameters are not set");
    if (N == 0) return SPGEMM_OK;
    k_mlp_forward<<<gridp(N), 256, 0, ctx->stream>>>(ctx->pred, X, N, pred);
    note_launch();
    SG_CUDA(ctx, cudaGetLastError());
    return SPGEMM_OK;
}

}  // extern "C"
