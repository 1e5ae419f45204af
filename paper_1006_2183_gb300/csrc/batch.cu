// Batched products in persistent launches.
#include "internal.cuh"

extern "C" {
spgemm_status_t spgemm_batch(spgemm_ctx_t ctx, int count, const spgemm_mat_t* A, const spgemm_mat_t* B,
                             spgemm_semiring_t sr, const spgemm_opts_t* opts, spgemm_mat_t* C) {
    (void)count; (void)A; (void)B; (void)sr; (void)opts; (void)C;
    return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "batch not built yet");
}
}
