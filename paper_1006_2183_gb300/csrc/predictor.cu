// Learned nnz(C(:,j)) predictor.
#include "internal.cuh"

extern "C" {
spgemm_status_t spgemm_predictor_set(spgemm_ctx_t ctx, const float* p) { (void)p; return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "todo"); }
spgemm_status_t spgemm_predictor_get(spgemm_ctx_t ctx, float* p) { (void)p; return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "todo"); }
spgemm_status_t spgemm_predictor_features(spgemm_ctx_t ctx, spgemm_mat_t A, spgemm_mat_t B, float* f, int64_t* n) {
    (void)A; (void)B; (void)f; (void)n; return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "todo"); }
spgemm_status_t spgemm_predictor_train_step(spgemm_ctx_t ctx, const float* X, const float* y, int64_t N, float lr,
                                            float* loss, float* grad) {
    (void)X; (void)y; (void)N; (void)lr; (void)loss; (void)grad; return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "todo"); }
spgemm_status_t spgemm_predictor_forward(spgemm_ctx_t ctx, const float* X, int64_t N, float* pred) {
    (void)X; (void)N; (void)pred; return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "todo"); }
}
