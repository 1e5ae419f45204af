// Host-side internals shared by the C-ABI translation units.
#pragma once
#include <cstdarg>
#include <cstdio>
#include <memory>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

struct spgemm_ctx {
    cudaStream_t stream = nullptr;
    spgemm_alloc_fn alloc = nullptr;
    spgemm_free_fn free_fn = nullptr;
    void* user = nullptr;
    int device = 0;
    std::string err;
    // learned predictor (device parameters + Adam moments)
    float* pred = nullptr;      // NPARAM
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* grad = nullptr;      // NPARAM (device gradient buffer)
    int adam_t = 0;
    bool pred_ready = false;
    // phase timing (CUDA events on the context stream)
    bool timing = false;
    int timing_quiet = 0;                // > 0: nested phases are not recorded (their parent is)
    struct Pending { int slot; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    int group = 0;
    double phase_ms[SPGEMM_NGROUP * 4 * SPGEMM_NPHASE] = {0};
    int64_t phase_cnt[SPGEMM_NGROUP * 4 * SPGEMM_NPHASE] = {0};
    // boolean semiring, set by a call that already knows it for every product it runs
    // (SUMMA checks its two operands once): -1 unknown, 0 no stored false value, 1 some
    int bool_hint = -1;
    // statistics of the last SUMMA call
    std::vector<int64_t> summa_stage_flops;
    int64_t summa_nonempty = 0;
    // Small device -> host reads (counts, offsets, flags) are written by a kernel into
    // mapped pinned memory and copied out on the host at the next sync_ctx: a
    // cudaMemcpyAsync device -> host would wait behind every bulk device -> host copy
    // already queued on the copy engine (from any stream, the caller's included).
    unsigned char* rb_host = nullptr;   // cudaHostAlloc(..., cudaHostAllocMapped)
    unsigned char* rb_dev = nullptr;    // its device address
    size_t rb_cap = 0, rb_used = 0;
    struct Readback { void* dst; size_t off, bytes; };
    std::vector<Readback> rb_pending;
};

// Shared ownership of an allocation (batch outputs share one buffer).
struct DevBuf {
    spgemm_ctx* ctx;
    void* p;
    DevBuf(spgemm_ctx* c, void* q) : ctx(c), p(q) {}
    ~DevBuf();
};

struct spgemm_mat {
    spgemm_ctx* ctx = nullptr;
    spgemm_format_t fmt = SPGEMM_FMT_CSC;
    spgemm_semiring_t sr = SPGEMM_PLUS_TIMES_F64;
    int64_t m = 0, n = 0, nnz = 0;   // logical dimensions (CSR: rows x cols of the matrix)
    // stored compressed arrays: CSC (and CSR as the CSC of the transpose)
    const int64_t* cp = nullptr;
    const int32_t* ir = nullptr;
    const void* num = nullptr;
    // DCSC extras
    int64_t nzc = 0;
    const int32_t* jc = nullptr;
    const int32_t* aux = nullptr;
    int64_t naux = 0, chunk = 1;
    std::vector<std::shared_ptr<DevBuf>> owned;
    bool checked = false;   // arrays passed the format check (library-made handles are born checked)
};

// One batched execution of products C_i = A_i * B_i over the item space
// (see kernels.cuh): analyze -> bin -> symbolic -> scan -> numeric.
struct Engine {
    spgemm_ctx* ctx = nullptr;
    spgemm_semiring_t sr = SPGEMM_PLUS_TIMES_F64;
    spgemm_opts_t opts;
    sg::TierCfg cfg;
    std::vector<sg::Prod> hprods;
    std::vector<int64_t> hitem_base;
    sg::Items it;
    std::vector<std::shared_ptr<DevBuf>> bufs;
    int64_t* flops = nullptr;
    uint8_t* bin = nullptr;
    int32_t* item_prod = nullptr;
    unsigned long long* ctr = nullptr;   // bin_count[NBIN], bin_cursor[NBIN], flops_total, slabs, store use, err,
                                         // store bound, false-value flag
    int64_t* bin_off_dev = nullptr;
    int2* list = nullptr;
    sg::DenseWork dw;                    // slab-tier state
    int64_t* nnz_item = nullptr;
    void* scan_tmp = nullptr;
    float* feat = nullptr;               // predictor inputs (items x 8) when requested
    int64_t* maxlen = nullptr;           // max_k nnz(A(:,k)) per item when requested
    std::shared_ptr<DevBuf> Coff_buf;    // item offsets (nitems + 1)
    int64_t* Coff = nullptr;
    int64_t bin_cnt[sg::NBIN] = {0};
    int64_t bin_off[sg::NBIN] = {0};
    // numeric lists of the hash tiers, binned by exact counts (set by the symbolic pass)
    uint8_t* nbin = nullptr;
    int2* nlist = nullptr;
    unsigned long long* nctr = nullptr;   // count[NBIN], cursor[NBIN]
    int64_t* nbin_off_dev = nullptr;
    int64_t nbin_cnt[sg::NBIN] = {0};
    int64_t nbin_off[sg::NBIN] = {0};
    bool numeric_bins = false;
    bool slab_rows_short = false;        // a column of the largest m would need > MAX_PARTS slabs
    int64_t flops_total = 0;
    int64_t nnz_total = -1;
    bool symbolic_done = false;
    bool want_prod_off = false;          // the symbolic pass also returns every product's first output
    std::vector<int64_t> prod_off;       // entry (nprod + 1 values, filled with nnz_total)
    int64_t overflow_items = 0;
};

struct spgemm_plan {
    spgemm_ctx* ctx = nullptr;
    spgemm_semiring_t sr;
    spgemm_opts_t opts;
    Engine E;
    spgemm_mat_t Aconv = nullptr, Bconv = nullptr;   // owned conversions (CSR inputs)
    int64_t m = 0, n = 0;          // output dimensions
    // batch plans
    bool is_batch = false;
    std::vector<spgemm_mat_t> convs;                 // owned conversions of batch operands
    std::vector<int64_t> pm, pn, colbase, outoff;    // per product: dims, colptr base, first entry
    std::shared_ptr<DevBuf> out_cp, out_r, out_v;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    ~spgemm_plan();
};

spgemm_status_t set_err(spgemm_ctx* ctx, spgemm_status_t s, const char* fmt, ...);

// Records CUDA events around a phase when the context has timing enabled.
struct PhaseTimer {
    spgemm_ctx* ctx;
    int phase;
    cudaEvent_t a = nullptr;
    PhaseTimer(spgemm_ctx* c, int ph, int sr) : ctx(c), phase((c->group * 4 + sr) * SPGEMM_NPHASE + ph) {
        if (ctx->timing && ctx->timing_quiet == 0) {
            cudaEventCreate(&a);
            cudaEventRecord(a, ctx->stream);
        }
    }
    ~PhaseTimer() {
        if (a) {
            cudaEvent_t b;
            cudaEventCreate(&b);
            cudaEventRecord(b, ctx->stream);
            ctx->pending.push_back({phase, a, b});
        }
    }
};
void* ctx_alloc(spgemm_ctx* ctx, size_t bytes);
void ctx_free(spgemm_ctx* ctx, void* p);
std::shared_ptr<DevBuf> ctx_buf(spgemm_ctx* ctx, size_t bytes);
size_t sr_size(spgemm_semiring_t sr);
sg::DMat dmat_of(const spgemm_mat* M);
spgemm_status_t check_cuda(spgemm_ctx* ctx, cudaError_t e, const char* what);
spgemm_status_t sync_ctx(spgemm_ctx* ctx);
// Queues a read of `bytes` at device address src into host memory dst, on the context
// stream; dst holds the bytes after the next sync_ctx (not before).
spgemm_status_t read_back(spgemm_ctx* ctx, void* dst, const void* src, size_t bytes);

// formats.cu
// Checks, in one launch and one synchronisation, every handle of `mats` that is a
// borrowed CSC/CSR not checked before (null entries and duplicates are skipped);
// SPGEMM_ERR_BAD_FORMAT names the first failing handle.  Passing handles are marked.
spgemm_status_t check_handles(spgemm_ctx* ctx, const std::vector<spgemm_mat*>& mats);
spgemm_status_t transpose_csc(spgemm_ctx* ctx, int64_t m, int64_t n, int64_t nnz, const int64_t* cp,
                              const int32_t* ir, const void* num, size_t w, spgemm_mat_t out_handle);
spgemm_status_t make_dcsc(spgemm_ctx* ctx, const spgemm_mat* csc, bool aux, spgemm_mat* out);
size_t radix_tmp_bytes(int64_t n);
void radix_sort_pairs(cudaStream_t st, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n, int bits,
                      void* tmp, bool* in_second);

// engine (api.cu)
spgemm_status_t engine_setup(Engine* E, spgemm_ctx* ctx, spgemm_semiring_t sr, const spgemm_opts_t& opts,
                             std::vector<sg::Prod> prods, bool want_features);
spgemm_status_t engine_symbolic(Engine* E);
spgemm_status_t engine_numeric(Engine* E, int32_t* Cir, void* Cv);
// predictor.cu: numeric pass without the symbolic pass of the hash tiers; returns C's arrays
spgemm_status_t engine_numeric_predicted(Engine* E, std::shared_ptr<DevBuf>* rbuf, std::shared_ptr<DevBuf>* vbuf);
// bounded.cu: numeric pass into min(flops, m) slots per hash-tier column (no symbolic pass
// for them); output is a CSC with gaps: column u in [col_start[u], col_end[u])
spgemm_status_t engine_numeric_bounded(Engine* E, std::shared_ptr<DevBuf>* rbuf, std::shared_ptr<DevBuf>* vbuf,
                                       std::shared_ptr<DevBuf>* colbuf, const int64_t** col_start,
                                       const int64_t** col_end);
// esc.cu: all products of E by expand-sort-compress (local rows); sets Coff and nnz_total
spgemm_status_t engine_esc(Engine* E, std::shared_ptr<DevBuf>* rbuf, std::shared_ptr<DevBuf>* vbuf);
// output arrays sized by the engine's nnz_total, values of the semiring width
spgemm_status_t engine_alloc_out(Engine* E, std::shared_ptr<DevBuf>* rbuf, std::shared_ptr<DevBuf>* vbuf);
sg::DMat csc_view(int64_t m, int64_t n, int64_t nnz, const int64_t* cp, const int32_t* ir, const void* num);
spgemm_mat_t new_owned_csc(spgemm_ctx* ctx, spgemm_semiring_t sr, int64_t m, int64_t n, int64_t nnz,
                           std::vector<std::shared_ptr<DevBuf>> owned, const int64_t* cp, const int32_t* ir,
                           const void* num);
spgemm_status_t to_csc_operand(spgemm_ctx* ctx, spgemm_mat_t M, spgemm_mat_t* conv, sg::DMat* d);

#define SG_STR2(x) #x
#define SG_STR(x) SG_STR2(x)
#define SG_WHERE __FILE_NAME__ ":" SG_STR(__LINE__)
#define SG_CUDA(ctx, call)                                                  \
    do {                                                                    \
        cudaError_t e__ = (call);                                           \
        if (e__ != cudaSuccess) return check_cuda((ctx), e__, #call " at " SG_WHERE); \
    } while (0)

#define SG_TRY(call)                               \
    do {                                           \
        spgemm_status_t s__ = (call);              \
        if (s__ != SPGEMM_OK) return s__;          \
    } while (0)
