// 2D Sparse SUMMA on a virtual g x g block grid (Sections 3.2, 3.5, 5.3).
#include "internal.cuh"

extern "C" {
spgemm_status_t spgemm_summa_blocked(spgemm_ctx_t ctx, spgemm_mat_t A, spgemm_mat_t B, int g,
                                     spgemm_semiring_t sr, const spgemm_opts_t* opts, spgemm_mat_t* C) {
    (void)A; (void)B; (void)g; (void)sr; (void)opts; (void)C;
    return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "summa not built yet");
}
spgemm_status_t spgemm_summa_stats(spgemm_ctx_t ctx, int64_t* stage_flops, int g, int64_t* nonempty) {
    (void)stage_flops; (void)g; (void)nonempty;
    return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "summa not built yet");
}
}
