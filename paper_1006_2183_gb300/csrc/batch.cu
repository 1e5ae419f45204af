// Many independent products in one execution: every product's columns join one
// item space, so each accumulator tier runs as a single grid-stride
// ("persistent") launch over a shared work list whatever the number and sizes
// of the products.  A batch plan keeps the analysis, the symbolic pass and the
// output arrays, and replays its numeric launches from a captured CUDA graph.
// The autotuner picks the tier thresholds by timing that numeric phase.
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>

#include "internal.cuh"

using namespace sg;

namespace {

spgemm_status_t collect_prods(spgemm_ctx* ctx, int count, const spgemm_mat_t* A, const spgemm_mat_t* B,
                              spgemm_semiring_t sr, std::vector<Prod>* prods, std::vector<spgemm_mat_t>* convs,
                              bool check = false) {
    if (count < 0 || (count > 0 && (!A || !B))) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "bad batch arrays");
    if (check) {
        std::vector<spgemm_mat*> ops;
        for (int i = 0; i < count; ++i) {
            if (!A[i] || !B[i]) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "null operand %d", i);
            ops.push_back(A[i]);
            ops.push_back(B[i]);
        }
        SG_TRY(check_handles(ctx, ops));
    }
    for (int i = 0; i < count; ++i) {
        if (!A[i] || !B[i]) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "null operand %d", i);
        if (A[i]->sr != sr || B[i]->sr != sr) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "semiring of pair %d", i);
        if (A[i]->n != B[i]->m) return set_err(ctx, SPGEMM_ERR_DIM_MISMATCH, "pair %d: inner dimensions differ", i);
        Prod pr;
        spgemm_mat_t ca = nullptr, cb = nullptr;
        SG_TRY(to_csc_operand(ctx, A[i], &ca, &pr.A));
        if (ca) convs->push_back(ca);
        SG_TRY(to_csc_operand(ctx, B[i], &cb, &pr.B));
        if (cb) convs->push_back(cb);
        prods->push_back(pr);
    }
    return SPGEMM_OK;
}

// Per-product column pointers and the first output entry of every product.
spgemm_status_t finish_outputs(struct spgemm_plan* P) {
    Engine& E = P->E;
    spgemm_ctx* ctx = P->ctx;
    const int64_t np = (int64_t)E.hprods.size();
    P->pm.resize(np);
    P->pn.resize(np);
    P->colbase.assign(np + 1, 0);
    for (int64_t i = 0; i < np; ++i) {
        P->pm[i] = E.hprods[i].A.m;
        P->pn[i] = E.hprods[i].B.n;
        P->colbase[i + 1] = P->colbase[i] + P->pn[i] + 1;
    }
    const int64_t total = P->colbase[np];
    if ((int64_t)E.prod_off.size() == np + 1) {
        // the symbolic pass returned where each product's output starts: no synchronisation
        P->outoff = E.prod_off;
        if (np == 1 && E.hprods[0].B.jc == nullptr) {
            // one product with a CSC B: the item offsets are C's column pointers
            P->out_cp = E.Coff_buf;
            return SPGEMM_OK;
        }
        P->out_cp = ctx_buf(ctx, 8 * std::max<int64_t>(total, 1) + 8 * (np + 1));
        if (!P->out_cp) return set_err(ctx, SPGEMM_ERR_OOM, "batch column pointers");
        int64_t* cp = (int64_t*)P->out_cp->p;
        int64_t* dcb = cp + std::max<int64_t>(total, 1);
        SG_CUDA(ctx, cudaMemcpyAsync(dcb, P->colbase.data(), 8 * (np + 1), cudaMemcpyHostToDevice, ctx->stream));
        launch_colptrs(ctx->stream, E.it, dcb, total, E.Coff, cp);
        // P->colbase must outlive the copy: it lives with the plan
        return SPGEMM_OK;
    }
    P->out_cp = ctx_buf(ctx, 8 * std::max<int64_t>(total, 1) + 8 * (2 * np + 2));
    if (!P->out_cp) return set_err(ctx, SPGEMM_ERR_OOM, "batch column pointers");
    int64_t* cp = (int64_t*)P->out_cp->p;
    int64_t* dcb = cp + std::max<int64_t>(total, 1);
    int64_t* doff = dcb + (np + 1);
    SG_CUDA(ctx, cudaMemcpyAsync(dcb, P->colbase.data(), 8 * (np + 1), cudaMemcpyHostToDevice, ctx->stream));
    launch_colptrs(ctx->stream, E.it, dcb, total, E.Coff, cp);
    launch_gather_offsets(ctx->stream, E.Coff, E.it.item_base, np, doff);
    P->outoff.assign(np + 1, 0);
    SG_TRY(read_back(ctx, P->outoff.data(), doff, 8 * (np + 1)));
    return sync_ctx(ctx);
}

spgemm_mat_t output_handle(struct spgemm_plan* P, int i, bool own) {
    const size_t w = sr_size(P->sr);
    const int64_t o = P->outoff[i];
    std::vector<std::shared_ptr<DevBuf>> owned;
    if (own) owned = {P->out_cp, P->out_r, P->out_v, P->E.Coff_buf};
    return new_owned_csc(P->ctx, P->sr, P->pm[i], P->pn[i], P->outoff[i + 1] - o, std::move(owned),
                         (const int64_t*)P->out_cp->p + P->colbase[i], (const int32_t*)P->out_r->p + o,
                         (const char*)P->out_v->p + w * o);
}

spgemm_status_t batch_plan_build(spgemm_ctx* ctx, int count, const spgemm_mat_t* A, const spgemm_mat_t* B,
                                 spgemm_semiring_t sr, const spgemm_opts_t& o, bool run_numeric,
                                 struct spgemm_plan* P) {
    P->ctx = ctx;
    P->sr = sr;
    P->opts = o;
    P->is_batch = true;
    std::vector<Prod> prods;
    SG_TRY(collect_prods(ctx, count, A, B, sr, &prods, &P->convs, o.check_inputs != 0));
    Engine& E = P->E;
    const bool learned = o.use_predictor && ctx->pred_ready && run_numeric;
    SG_TRY(engine_setup(&E, ctx, sr, o, prods, learned));
    E.want_prod_off = true;
    if (learned) {
        SG_TRY(engine_numeric_predicted(&E, &P->out_r, &P->out_v));
    } else {
        SG_TRY(engine_symbolic(&E));
        SG_TRY(engine_alloc_out(&E, &P->out_r, &P->out_v));
        if (run_numeric) SG_TRY(engine_numeric(&E, (int32_t*)P->out_r->p, P->out_v->p));
    }
    return finish_outputs(P);
}

template <class SR>
void numeric_launches(struct spgemm_plan* P) {
    Engine& E = P->E;
    const bool nb = E.numeric_bins;   // hash tiers binned by exact counts
    launch_numeric<SR>(P->ctx->stream, E.it, E.cfg, nb ? E.nlist : E.list, nb ? E.nbin_off : E.bin_off,
                       nb ? E.nbin_cnt : E.bin_cnt, E.dw, E.Coff, (int32_t*)P->out_r->p,
                       (typename SR::T*)P->out_v->p, 1);
    launch_numeric<SR>(P->ctx->stream, E.it, E.cfg, E.list, E.bin_off, E.bin_cnt, E.dw, E.Coff,
                       (int32_t*)P->out_r->p, (typename SR::T*)P->out_v->p, 2);
}

void all_numeric_launches(struct spgemm_plan* P) {
    switch (P->sr) {
    case SPGEMM_PLUS_TIMES_F64: numeric_launches<PT64>(P); break;
    case SPGEMM_MIN_PLUS_F32: numeric_launches<MP32>(P); break;
    case SPGEMM_OR_AND_BOOL: numeric_launches<BOOL8>(P); break;
    case SPGEMM_PLUS_TIMES_I64: numeric_launches<PTI64>(P); break;
    }
}

struct TuneKey {
    int sr, count, lgflops;
    bool operator<(const TuneKey& o) const {
        return std::tie(sr, count, lgflops) < std::tie(o.sr, o.count, o.lgflops);
    }
};
std::map<std::pair<spgemm_ctx*, TuneKey>, std::tuple<int, int, int, int>> g_tune_cache;

// Device time of whole spgemm_batch calls with opts o (one warm-up, then the best of two).
float time_batch_calls(spgemm_ctx* ctx, int count, const spgemm_mat_t* A, const spgemm_mat_t* B,
                       spgemm_semiring_t sr, const spgemm_opts_t& o, spgemm_status_t* st) {
    std::vector<spgemm_mat_t> C(std::max(count, 1), nullptr);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    *st = SPGEMM_OK;
    for (int r = 0; r < 3 && *st == SPGEMM_OK; ++r) {
        cudaEventRecord(e0, ctx->stream);
        *st = spgemm_batch(ctx, count, A, B, sr, &o, C.data());
        cudaEventRecord(e1, ctx->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) best = std::min(best, ms);
        if (*st == SPGEMM_OK)
            for (int i = 0; i < count; ++i) spgemm_mat_destroy(C[i]);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace

extern "C" {

spgemm_status_t spgemm_batch(spgemm_ctx_t ctx, int count, const spgemm_mat_t* A, const spgemm_mat_t* B,
                             spgemm_semiring_t sr, const spgemm_opts_t* opts, spgemm_mat_t* C) {
    if (!ctx || (count > 0 && !C)) return SPGEMM_ERR_INVALID_ARG;
    if ((int)sr < 0 || (int)sr > 3) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "bad semiring");
    spgemm_opts_t o;
    spgemm_opts_default(&o);
    if (opts) o = *opts;
    std::unique_ptr<struct spgemm_plan> P(new struct spgemm_plan());
    SG_TRY(batch_plan_build(ctx, count, A, B, sr, o, true, P.get()));
    for (int i = 0; i < count; ++i) C[i] = output_handle(P.get(), i, true);
    return SPGEMM_OK;
}

spgemm_status_t spgemm_batch_plan(spgemm_ctx_t ctx, int count, const spgemm_mat_t* A, const spgemm_mat_t* B,
                                  spgemm_semiring_t sr, const spgemm_opts_t* opts, spgemm_plan_t* plan) {
    if (!ctx || !plan) return SPGEMM_ERR_INVALID_ARG;
    if ((int)sr < 0 || (int)sr > 3) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "bad semiring");
    spgemm_opts_t o;
    spgemm_opts_default(&o);
    if (opts) o = *opts;
    o.use_predictor = 0;   // the plan keeps exact offsets for replays
    auto* P = new struct spgemm_plan();
    spgemm_status_t s = batch_plan_build(ctx, count, A, B, sr, o, false, P);
    if (s != SPGEMM_OK) {
        delete P;
        return s;
    }
    *plan = P;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_batch_execute(spgemm_plan_t P) {
    if (!P || !P->is_batch) return SPGEMM_ERR_INVALID_ARG;
    spgemm_ctx* ctx = P->ctx;
    if (ctx->stream == nullptr) {
        // the legacy default stream cannot be captured: launch directly
        PhaseTimer t(ctx, SPGEMM_PHASE_NUMERIC_HASH, P->sr);
        all_numeric_launches(P);
        SG_CUDA(ctx, cudaGetLastError());
        return SPGEMM_OK;
    }
    if (!P->gexec) {
        // capture the numeric launches once (no allocation or host sync inside)
        const bool timing = ctx->timing;
        ctx->timing = false;
        // one eager run first: it sets the kernels' shared-memory attributes outside the capture
        all_numeric_launches(P);
        SG_CUDA(ctx, cudaGetLastError());
        SG_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        all_numeric_launches(P);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
        ctx->timing = timing;
        if (e != cudaSuccess) return check_cuda(ctx, e, "cudaStreamEndCapture");
        P->graph = g;
        SG_CUDA(ctx, cudaGraphInstantiate(&P->gexec, g, 0));
        return SPGEMM_OK;
    }
    PhaseTimer t(ctx, SPGEMM_PHASE_NUMERIC_HASH, P->sr);
    SG_CUDA(ctx, cudaGraphLaunch(P->gexec, ctx->stream));
    note_launch();
    return SPGEMM_OK;
}

spgemm_status_t spgemm_batch_outputs(spgemm_plan_t P, spgemm_mat_t* C) {
    if (!P || !P->is_batch || !C) return SPGEMM_ERR_INVALID_ARG;
    for (size_t i = 0; i < P->pm.size(); ++i) C[i] = output_handle(P, (int)i, false);
    return SPGEMM_OK;
}

spgemm_status_t spgemm_autotune(spgemm_ctx_t ctx, int count, const spgemm_mat_t* A, const spgemm_mat_t* B,
                                spgemm_semiring_t sr, spgemm_opts_t* opts) {
    if (!ctx || !opts) return SPGEMM_ERR_INVALID_ARG;
    int64_t fl = 0;
    {
        // total flops class of the batch
        std::unique_ptr<struct spgemm_plan> P(new struct spgemm_plan());
        P->ctx = ctx;
        std::vector<Prod> prods;
        SG_TRY(collect_prods(ctx, count, A, B, sr, &prods, &P->convs));
        SG_TRY(engine_setup(&P->E, ctx, sr, *opts, prods, false));
        fl = P->E.flops_total;
    }
    int lg = 0;
    while ((int64_t(1) << lg) < fl && lg < 62) ++lg;
    const bool try_pred = opts->use_predictor != 0 && ctx->pred_ready;
    TuneKey key{(int)sr * 2 + (try_pred ? 1 : 0), count, lg};
    auto hit = g_tune_cache.find({ctx, key});
    if (hit == g_tune_cache.end()) {
        const int warp_c[] = {128, 512};
        const int block_c[] = {1024, 4096};
        const int part_c[] = {32768, 262144};
        double best = 1e30;
        std::tuple<int, int, int, int> pick{opts->warp_max_flops, opts->block_max_flops, opts->dense_part_flops, 0};
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int wm : warp_c)
            for (int bm : block_c)
                for (int pf : part_c) {
                    spgemm_opts_t o = *opts;
                    o.warp_max_flops = wm;
                    o.block_max_flops = bm;
                    o.dense_part_flops = pf;
                    spgemm_plan_t P = nullptr;
                    SG_TRY(spgemm_batch_plan(ctx, count, A, B, sr, &o, &P));
                    std::unique_ptr<struct spgemm_plan> hold(P);
                    SG_TRY(spgemm_batch_execute(P));   // capture
                    float ms = 0.f, tot = 0.f;
                    for (int r = 0; r < 3; ++r) {
                        cudaEventRecord(e0, ctx->stream);
                        SG_TRY(spgemm_batch_execute(P));
                        cudaEventRecord(e1, ctx->stream);
                        cudaEventSynchronize(e1);
                        cudaEventElapsedTime(&ms, e0, e1);
                        tot += ms;
                    }
                    if (tot < best) {
                        best = tot;
                        pick = {wm, bm, pf, 0};
                    }
                }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        {
            // the grid above times the numeric pass alone; the thresholds also move work
            // between the counting passes, so the pick must beat the caller's own
            // thresholds as whole calls, or the caller's are kept
            spgemm_opts_t o = *opts;
            o.use_predictor = 0;
            spgemm_status_t s0, s1;
            const float t_given = time_batch_calls(ctx, count, A, B, sr, o, &s0);
            SG_TRY(s0);
            o.warp_max_flops = std::get<0>(pick);
            o.block_max_flops = std::get<1>(pick);
            o.dense_part_flops = std::get<2>(pick);
            const float t_pick = time_batch_calls(ctx, count, A, B, sr, o, &s1);
            SG_TRY(s1);
            if (t_given <= t_pick) pick = {opts->warp_max_flops, opts->block_max_flops, opts->dense_part_flops, 0};
        }
        if (try_pred) {
            // the predictor replaces the symbolic pass of the hash tiers but adds its own launches
            // and a move of C: keep it only where the whole batched call measured faster with it
            spgemm_opts_t o = *opts;
            o.warp_max_flops = std::get<0>(pick);
            o.block_max_flops = std::get<1>(pick);
            o.dense_part_flops = std::get<2>(pick);
            spgemm_status_t s1, s0;
            o.use_predictor = 1;
            const float t1 = time_batch_calls(ctx, count, A, B, sr, o, &s1);
            SG_TRY(s1);
            o.use_predictor = 0;
            const float t0 = time_batch_calls(ctx, count, A, B, sr, o, &s0);
            SG_TRY(s0);
            std::get<3>(pick) = t1 < t0 ? 1 : 0;
        }
        hit = g_tune_cache.emplace(std::make_pair(ctx, key), pick).first;
    }
    opts->warp_max_flops = std::get<0>(hit->second);
    opts->block_max_flops = std::get<1>(hit->second);
    opts->dense_part_flops = std::get<2>(hit->second);
    if (try_pred) opts->use_predictor = std::get<3>(hit->second);
    return SPGEMM_OK;
}

}  // extern "C"
