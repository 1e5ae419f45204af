/*
 * spgemm.h -- C ABI of the GB300 semiring SpGEMM library (libspgemm.so).
 *
 * Computes C = A*B over a semiring (Section 1: "the product of two sparse
 * matrices (SpGEMM) over a semiring"), column by column (Gustavson's
 * formulation, Section 2.1), including the hypersparse DCSC block products and
 * stage-wise merges of 2D Sparse SUMMA (Sections 2.3, 3.2, 3.5) run as a
 * virtual g x g block grid on one GPU.
 *
 * Conventions for every entry point
 *   - Indices are 0-based.  Matrices are CSC: int64 column pointers (n+1),
 *     int32 row indices sorted strictly ascending inside each column, values
 *     of the semiring's element type (double / float / uint8 / int64).
 *   - Every pointer passed in a matrix handle is a DEVICE pointer on the
 *     context's GPU, unless an entry point says otherwise.
 *   - All work is enqueued on the context's CUDA stream.  The product calls
 *     synchronise that stream where a host decision needs a device count, so a
 *     product call returns with its result complete; handle creation and export
 *     do not synchronise.  The counts a flat product waits for: the input check
 *     (once per borrowed handle), the column count of every accumulator tier
 *     (launch sizes and list offsets), the slab count and row-set bound of the
 *     long columns (their arrays), the output size nnz(C) (the allocation of
 *     C), and, with the predictor, the predicted capacity and the overflowed
 *     columns.  SUMMA adds the block layouts of the split and of every merge.
 *   - Every function returns spgemm_status_t and never aborts; the message of
 *     the last failure is available from spgemm_last_error(ctx).
 *   - Results are structural: C(i,j) exists iff some k pairs a stored A(i,k)
 *     with a stored B(k,j); entries whose value equals the semiring zero are
 *     kept.  C's rows are sorted ascending within each column.  For the three
 *     exact semirings the result is bit-identical whatever the options
 *     (predictor on/off, batching, grid size g, tier thresholds).
 *
 * Ownership
 *   - Input handles made by spgemm_mat_csc / spgemm_mat_csr BORROW the
 *     caller's arrays and never free them; the caller keeps them alive until
 *     the handle is destroyed.
 *   - Handles returned by the library (products, conversions) OWN arrays
 *     allocated through the context allocator; spgemm_mat_destroy frees them.
 *   - Temporaries are allocated through the context allocator for the
 *     duration of one call (freed in stream order on the context stream before
 *     it returns); the predictor's parameters live until spgemm_ctx_destroy.
 *     spgemm_colptr_noalloc allocates nothing.
 */
#ifndef SPGEMM_H
#define SPGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPGEMM_OK = 0,
    SPGEMM_ERR_INVALID_ARG = 1,    /* null pointer, negative size, bad enum value      */
    SPGEMM_ERR_DIM_MISMATCH = 2,   /* inner dimensions of A and B differ               */
    SPGEMM_ERR_BAD_FORMAT = 3,     /* colptr not monotone, row out of range/unsorted   */
    SPGEMM_ERR_OOM = 4,            /* the allocator returned NULL                      */
    SPGEMM_ERR_INDEX_OVERFLOW = 5, /* a row count or dimension beyond int32 rows       */
    SPGEMM_ERR_TIMEOUT = 6,        /* a bounded device wait gave up                    */
    SPGEMM_ERR_CUDA = 7,           /* a CUDA runtime call failed                       */
    SPGEMM_ERR_UNSUPPORTED = 8,    /* combination not implemented                      */
    SPGEMM_ERR_STATE = 9           /* call out of order (e.g. numeric before symbolic) */
} spgemm_status_t;

/* The four semirings (Section 1 names SpGEMM over an arbitrary semiring). */
typedef enum {
    SPGEMM_PLUS_TIMES_F64 = 0, /* (+, *, 0) on double                                  */
    SPGEMM_MIN_PLUS_F32 = 1,   /* (min, +, +inf) on float; fl32(a+b), round to nearest  */
    SPGEMM_OR_AND_BOOL = 2,    /* (or, and, false) on uint8, nonzero byte = true        */
    SPGEMM_PLUS_TIMES_I64 = 3  /* (+, *, 0) on int64, two's-complement wraparound       */
} spgemm_semiring_t;

typedef enum {
    SPGEMM_FMT_CSC = 0,  /* Section 2.2, Fig. 5                                          */
    SPGEMM_FMT_CSR = 1,  /* rows compressed; stored as the CSC of the transpose          */
    SPGEMM_FMT_DCSC = 2  /* Section 2.3: JC, CP, IR, NUM (+ AUX column index)            */
} spgemm_format_t;

typedef struct spgemm_ctx* spgemm_ctx_t;
typedef struct spgemm_mat* spgemm_mat_t;
typedef struct spgemm_plan* spgemm_plan_t;

/* Device allocator callbacks: alloc(bytes, user) returns a device pointer or
 * NULL; free(ptr, user).  Both are called on the host thread that makes the
 * library call, in stream order of the context stream. */
typedef void* (*spgemm_alloc_fn)(size_t bytes, void* user);
typedef void (*spgemm_free_fn)(void* ptr, void* user);

/* Options.  spgemm_opts_default fills the defaults; a NULL opts pointer means
 * defaults everywhere. */
typedef struct {
    int use_predictor;        /* 1: size outputs from the learned nnz predictor and skip
                                 the exact symbolic pass; overflowed columns are redone
                                 exactly, so the result is unchanged.  Default 0.      */
    int summa_fused;          /* reserved, must be 0: spgemm_summa_blocked always
                                 materialises each stage's partial products and merges
                                 them (SPGEMM_ERR_UNSUPPORTED otherwise).              */
    int summa_merge_every;    /* staged mode: merge after this many stages (0 = after
                                 the last stage, the paper's buffered triples).        */
    int warp_max_flops;       /* columns with flops <= this use warp-wide hash tables  */
    int block_max_flops;      /* columns with flops <= this use CTA-wide hash tables;
                                 longer columns (the slab tier) are cut into row slabs,
                                 each counted and then accumulated by one CTA (at most
                                 4096).  -1 (default) = automatic: 4096 for operands of
                                 at most 32768 rows, 1024 for larger ones.            */
    int dense_part_flops;     /* slab tier: target flops per row slab of a long column
                                 (default 65536); a column whose B column is long gets
                                 fewer, larger slabs                                    */
    float predictor_margin;   /* capacity = (1 + margin) * prediction (+ slack)        */
    int range_table_slots;    /* ignored (kept for the layout of this struct)          */
    int block_kernel;         /* spgemm_summa_blocked stage products: 0 = the column
                                 tiers (default), 1 = expand-sort-compress, the
                                 data-parallel form of the outer-product multiply of
                                 Section 2.4 (needs < 2^32 products per merge group) */
    int range_slab_rows;      /* long columns: most rows of one row slab (its row
                                 bitmap lives in shared memory), rounded to a
                                 multiple of 32 and clamped to [4096, 2^20]; raised
                                 where a column would need more than 64 slabs.
                                 0 = default (2^19).  A long column of more than
                                 64 * (2^20 - 32) rows is SPGEMM_ERR_UNSUPPORTED.   */
    int check_inputs;         /* 1 (default): every product call first checks, on the
                                 device, each borrowed CSC/CSR operand it has not checked
                                 before (the spgemm_mat_validate invariants) and returns
                                 SPGEMM_ERR_BAD_FORMAT before any product kernel runs; a
                                 handle passes once and is then trusted (re-check arrays
                                 changed in place with spgemm_mat_validate).  0: skip. */
    int reserved[4];
} spgemm_opts_t;

void spgemm_opts_default(spgemm_opts_t* opts);

/* ---------------------------------------------------------------- context */
/* stream: a cudaStream_t (NULL = legacy default stream).  alloc/free may be NULL,
 * in which case cudaMallocAsync/cudaFreeAsync on the stream are used.
 * Where a call waits for the device (the counts behind C's size, flags), it reads
 * those few bytes through mapped pinned host memory written by a kernel on the
 * context's stream, not with a device-to-host cudaMemcpy: such a copy waits behind
 * every bulk device-to-host copy already queued on the copy engine, the caller's
 * included, so a caller may copy one result back on another stream while the next
 * product runs.  The context holds that buffer (64 KiB or more) until
 * spgemm_ctx_destroy. */
spgemm_status_t spgemm_ctx_create(spgemm_ctx_t* ctx, void* cuda_stream, spgemm_alloc_fn alloc,
                                  spgemm_free_fn free_fn, void* alloc_user);
spgemm_status_t spgemm_ctx_destroy(spgemm_ctx_t ctx);
spgemm_status_t spgemm_ctx_set_stream(spgemm_ctx_t ctx, void* cuda_stream);
const char* spgemm_last_error(spgemm_ctx_t ctx);
const char* spgemm_status_string(spgemm_status_t s);

/* ---------------------------------------------------------------- matrices */
/* Borrowing CSC handle over device arrays (Section 2.2, Fig. 5): colptr[n+1]
 * int64, rowidx[nnz] int32, vals[nnz] of the semiring type (vals may be NULL
 * for a pattern-only matrix, read as all-ones / all-true / zero for min-plus).
 * No device work is done here: the arrays are checked by the first product
 * call that uses the handle (check_inputs) or by spgemm_mat_validate. */
spgemm_status_t spgemm_mat_csc(spgemm_ctx_t ctx, spgemm_mat_t* out, int64_t m, int64_t n, int64_t nnz,
                               const int64_t* colptr, const int32_t* rowidx, const void* vals,
                               spgemm_semiring_t semiring);
/* Borrowing CSR handle: rowptr[m+1], colidx[nnz] sorted within each row. */
spgemm_status_t spgemm_mat_csr(spgemm_ctx_t ctx, spgemm_mat_t* out, int64_t m, int64_t n, int64_t nnz,
                               const int64_t* rowptr, const int32_t* colidx, const void* vals,
                               spgemm_semiring_t semiring);
/* Checks the CSC/CSR invariants on the device: colptr[0] == 0, colptr
 * monotone, colptr[n] == nnz, rows in [0, m) and strictly ascending per column.
 * Returns SPGEMM_ERR_BAD_FORMAT on a violation (synchronises); on success the
 * handle is marked checked (see spgemm_opts_t.check_inputs). */
spgemm_status_t spgemm_mat_validate(spgemm_mat_t mat);
/* CSC -> DCSC (Section 2.3): JC = ids of the nzc nonempty columns, CP = their
 * pointers (nzc+1), IR/NUM shared with the source (the result borrows them, so
 * the source must outlive it).  With build_aux, AUX is built over chunks of
 * ceil(n/nzc) columns: AUX[t] = position in JC of the first nonzero column with
 * id >= t*chunk, last entry nzc (the paper leaves empty chunks unspecified;
 * this reading makes chunk t's columns JC[AUX[t] .. AUX[t+1])). */
spgemm_status_t spgemm_mat_to_dcsc(spgemm_ctx_t ctx, spgemm_mat_t csc, int build_aux, spgemm_mat_t* out);
/* Transpose (Section 2.4 transposes B once): CSC of A^T, rows sorted.  Owns its arrays. */
spgemm_status_t spgemm_mat_transpose(spgemm_ctx_t ctx, spgemm_mat_t a, spgemm_mat_t* out);
/* Permuted copy B = P A Q^T, B(row_perm[i], col_perm[j]) = A(i, j) (the random
 * symmetric permutation of Section 5.3.3 relabels vertices so that
 * C' = (PAP^T)(PBP^T) = PCP^T balances the 2D grid).  row_perm (m entries) and
 * col_perm (n entries) are device int32 arrays, each a permutation; NULL means
 * the identity.  A is CSC or CSR.  Result: CSC, rows sorted, owning its arrays.
 * Errors: INVALID_ARG when an array is not a permutation (checked on the device;
 * synchronises the stream), UNSUPPORTED for DCSC, INDEX_OVERFLOW for nnz >= 2^32. */
spgemm_status_t spgemm_mat_permute(spgemm_ctx_t ctx, spgemm_mat_t a, const int32_t* row_perm,
                                   const int32_t* col_perm, spgemm_mat_t* out);
/* Read back a handle's shape and device arrays.  For DCSC, colptr is CP,
 * jc/aux/nzc/chunk describe the compressed column index (NULL outputs are
 * skipped).  Pointers stay owned by the handle. */
spgemm_status_t spgemm_mat_export(spgemm_mat_t mat, int64_t* m, int64_t* n, int64_t* nnz,
                                  const int64_t** colptr, const int32_t** rowidx, const void** vals);
spgemm_status_t spgemm_mat_export_dcsc(spgemm_mat_t mat, int64_t* nzc, const int32_t** jc,
                                       const int32_t** aux, int64_t* naux, int64_t* chunk);
spgemm_status_t spgemm_mat_format(spgemm_mat_t mat, spgemm_format_t* fmt, spgemm_semiring_t* sr);
spgemm_status_t spgemm_mat_destroy(spgemm_mat_t mat);

/* ---------------------------------------------------------------- measurement */
/* Phases timed with CUDA events on the context stream when timing is enabled. */
#define SPGEMM_NPHASE 8
typedef enum {
    SPGEMM_PHASE_ANALYZE = 0,        /* flops per column, binning, dense work items     */
    SPGEMM_PHASE_SYMBOLIC_HASH = 1,  /* symbolic pass, hash-table tiers                 */
    SPGEMM_PHASE_SYMBOLIC_DENSE = 2, /* symbolic pass, long columns (ranges / dense)    */
    SPGEMM_PHASE_SCAN = 3,           /* column pointers of C                            */
    SPGEMM_PHASE_NUMERIC_HASH = 4,   /* numeric pass, hash-table tiers                  */
    SPGEMM_PHASE_NUMERIC_DENSE = 5,  /* numeric pass, long columns (ranges / dense)     */
    SPGEMM_PHASE_PREDICT = 6,        /* predictor inference + overflow repair           */
    SPGEMM_PHASE_MERGE = 7           /* SUMMA stage merge                               */
} spgemm_phase_t;
#define SPGEMM_NGROUP 4
/* Enable (1) / disable (0) phase timing; enabling resets the accumulators. */
spgemm_status_t spgemm_ctx_timing(spgemm_ctx_t ctx, int enable);
/* Label the phases timed from now on with a caller-chosen group in
 * [0, SPGEMM_NGROUP) (e.g. one group per kind of product); default 0. */
spgemm_status_t spgemm_ctx_timing_group(spgemm_ctx_t ctx, int group);
/* Accumulated milliseconds and counts per (group, semiring, phase) since timing
 * was enabled (synchronises the stream).  ms and count each hold
 * SPGEMM_NGROUP * 4 * SPGEMM_NPHASE entries, indexed
 * [(group * 4 + semiring) * SPGEMM_NPHASE + phase]. */
spgemm_status_t spgemm_ctx_phase_ms(spgemm_ctx_t ctx, double* ms, int64_t* count);
/* Number of kernels this library has launched in the process so far. */
int64_t spgemm_launch_count(void);

/* ---------------------------------------------------------------- flat product */
/* Plan C = A*B (A: m x k, B: k x n; CSC, CSR or DCSC operands): per-column flops
 * flops_j = sum over k in B(:,j) of nnz(A(:,k)) (Section 1's "flops"), predictor
 * features when enabled, and the binning of columns into accumulator tiers.
 * Errors: DIM_MISMATCH when A.n != B.m, INVALID_ARG for semiring mismatch. */
spgemm_status_t spgemm_plan(spgemm_ctx_t ctx, spgemm_mat_t A, spgemm_mat_t B, spgemm_semiring_t semiring,
                            const spgemm_opts_t* opts, spgemm_plan_t* plan);
/* Exact symbolic pass: nnz(C(:,j)) = |union of the row sets of A(:,k), k in B(:,j)|
 * and C's column pointers; writes the total to *nnz_C (synchronises).  With the
 * predictor enabled this call is optional: spgemm_numeric then sizes C from the
 * predictions and repairs mispredicted columns exactly. */
spgemm_status_t spgemm_symbolic(spgemm_plan_t plan, int64_t* nnz_C);
/* Numeric pass: C(:,j) = (+)_{k in B(:,j)} A(:,k) (x) B(k,j), rows sorted; C is
 * a new owning CSC handle (m x n).  Runs the symbolic pass first if it has not
 * run and the predictor is off. */
spgemm_status_t spgemm_numeric(spgemm_plan_t plan, spgemm_mat_t* C);
/* Plan statistics: total flops, nnz(C) (after numeric), columns per tier,
 * predictor overflow count.  Any output pointer may be NULL. */
spgemm_status_t spgemm_plan_stats(spgemm_plan_t plan, int64_t* flops, int64_t* nnz_C, int64_t* tier_cols4,
                                  int64_t* overflow_cols);
/* Per-tier totals of the plan: columns, flops, nnz(C) (after the symbolic pass,
 * else -1) and nnz of the B columns, for tiers {empty, warp hash, CTA hash,
 * dense}; any pointer may be NULL. */
spgemm_status_t spgemm_plan_tier_stats(spgemm_plan_t plan, int64_t* cols4, int64_t* flops4, int64_t* nnz4,
                                       int64_t* bnnz4);
spgemm_status_t spgemm_plan_destroy(spgemm_plan_t plan);

/* One-call product: plan + symbolic + numeric. */
spgemm_status_t spgemm_multiply(spgemm_ctx_t ctx, spgemm_mat_t A, spgemm_mat_t B, spgemm_semiring_t semiring,
                                const spgemm_opts_t* opts, spgemm_mat_t* C);

/* ---------------------------------------------------------------- 2D Sparse SUMMA */
/* C = A*B on a virtual g x g grid (Sections 3.2 and 3.5; single-processor
 * simulation as in Section 5.3): A and B are split into g x g blocks of
 * ceil(dim/g) rows/columns (the last block may be short or empty), each block
 * stored as DCSC with AUX; stage s computes the hypersparse block products
 * A_{I,s} * B_{s,J} for all I, J and the stage partials are merged into C_{IJ}
 * (Section 6.1 buffers the partial triples and merges them later).  Returns
 * the flat CSC C (m x n), identical in structure to spgemm_multiply.
 * Errors as spgemm_plan; INVALID_ARG for g < 1. */
spgemm_status_t spgemm_summa_blocked(spgemm_ctx_t ctx, spgemm_mat_t A, spgemm_mat_t B, int g,
                                     spgemm_semiring_t semiring, const spgemm_opts_t* opts, spgemm_mat_t* C);
/* The same product with the stage merges on a second stream (Sections 7.2-7.3:
 * overlap each stage's data movement with the local work; on one GPU the
 * overlap is between the merge of one group of summa_merge_every stages and the
 * stage products of the next group).  Stage products run on ctx's stream from
 * the calling thread; merges run on merge_ctx's stream from a worker thread the
 * library starts and joins within this call, so merge_ctx's allocator callbacks
 * are called from that thread and must be thread-safe.  ctx's callbacks stay on
 * the calling thread.  The result is identical to spgemm_summa_blocked with the
 * same opts (for plus-times FP64 up to summation order) and is allocated
 * through merge_ctx, which must outlive it.  Both contexts must be on the same
 * device; the call returns after both streams have finished its work.
 * INVALID_ARG if merge_ctx is NULL, equal to ctx or on another device; other
 * errors as spgemm_summa_blocked (a merge error is reported on ctx). */
spgemm_status_t spgemm_summa_pipelined(spgemm_ctx_t ctx, spgemm_ctx_t merge_ctx, spgemm_mat_t A, spgemm_mat_t B,
                                       int g, spgemm_semiring_t semiring, const spgemm_opts_t* opts,
                                       spgemm_mat_t* C);
/* Block statistics of the last summa call on this context: per-stage flops
 * (g entries) and the number of nonempty block products.  Outputs may be NULL. */
spgemm_status_t spgemm_summa_stats(spgemm_ctx_t ctx, int64_t* stage_flops, int g, int64_t* nonempty_products);
/* Work of every block product of the virtual grid, without computing it:
 * flops[(s*g + J)*g + I] = flops(A_{I,s} * B_{s,J}) (multiply count), for the
 * load-imbalance measure of Section 7.1 (max over processors / mean, per stage
 * and over all stages).  flops is a host array of g*g*g int64; A and B as for
 * spgemm_summa_blocked (only the structure is used).  Synchronises the stream. */
spgemm_status_t spgemm_summa_block_flops(spgemm_ctx_t ctx, spgemm_mat_t A, spgemm_mat_t B, int g, int64_t* flops);

/* ---------------------------------------------------------------- batching */
/* count independent products C[i] = A[i]*B[i] (all over one semiring) in one
 * plan: the columns of every product are binned together and each tier runs
 * as one persistent launch over a shared work queue; with opts->use_predictor
 * the symbolic pass is skipped as in spgemm_numeric.  C[i] are owning CSC
 * handles (they share one allocation, freed with the last of them). */
spgemm_status_t spgemm_batch(spgemm_ctx_t ctx, int count, const spgemm_mat_t* A, const spgemm_mat_t* B,
                             spgemm_semiring_t semiring, const spgemm_opts_t* opts, spgemm_mat_t* C);

/* Reusable batch: analysis, symbolic pass and output allocation once; then
 * spgemm_batch_execute recomputes every C[i]'s values from the current values
 * of the A[i], B[i] arrays (same structure, same device pointers).  The numeric
 * launches are captured into a CUDA graph on the first execute and replayed
 * after that (on the legacy default stream, which cannot be captured, they are
 * launched directly every time).  spgemm_batch_outputs returns handles that borrow the plan's
 * arrays (valid until spgemm_plan_destroy). */
spgemm_status_t spgemm_batch_plan(spgemm_ctx_t ctx, int count, const spgemm_mat_t* A, const spgemm_mat_t* B,
                                  spgemm_semiring_t semiring, const spgemm_opts_t* opts, spgemm_plan_t* plan);
spgemm_status_t spgemm_batch_execute(spgemm_plan_t plan);
spgemm_status_t spgemm_batch_outputs(spgemm_plan_t plan, spgemm_mat_t* C);
/* Autotuner: times the numeric phase of the batch for a small set of tier
 * thresholds (warp_max_flops, block_max_flops, dense_part_flops), then times
 * whole spgemm_batch calls with the fastest of them and with the thresholds
 * *opts came with, and writes the faster pair's thresholds into *opts (the
 * thresholds also move work between the counting passes, which the numeric
 * timing does not see).  When opts->use_predictor is set and the context holds
 * predictor parameters, it then times whole spgemm_batch calls with and
 * without the predictor (at the chosen thresholds) and leaves use_predictor at
 * 1 only if the predictor measured faster, so the tuned call never loses to
 * the exact symbolic pass.  Other fields are kept.  Results are cached in the
 * context per (semiring, predictor tried, number of products, total flops
 * rounded to a power of two). */
spgemm_status_t spgemm_autotune(spgemm_ctx_t ctx, int count, const spgemm_mat_t* A, const spgemm_mat_t* B,
                                spgemm_semiring_t semiring, spgemm_opts_t* opts);

/* ---------------------------------------------------------------- no device allocation */
/* Column pointers of C = A*B (C's structure: Ccolptr[0] = 0, Ccolptr[j+1] -
 * Ccolptr[j] = nnz(C(:,j))) computed without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory where they need C's structure -- programs that
 * give the library a fixed, pre-planned memory budget, latency-critical paths
 * where an allocation call and the synchronisation it can cause are not
 * allowed, or plugins inside a host program whose memory manager owns all
 * device memory.  Everything it touches is either the caller's (A, B as device
 * CSC arrays of an m x k and a k x n matrix; Ccolptr, n+1 int64 on the device,
 * written) or one file-scope device array of SPGEMM_NOALLOC_MAX_TILES int64
 * (32 KiB, resident on every GPU that loads the library until the process
 * exits).  Limits: m <= SPGEMM_NOALLOC_MAX_ROWS (a bitmap of m bits lives in
 * shared memory) and n <= SPGEMM_NOALLOC_MAX_TILES * 4096; larger inputs return
 * SPGEMM_ERR_UNSUPPORTED without launching anything.  Work is enqueued on
 * cuda_stream (a cudaStream_t; NULL = legacy default stream) and the call does
 * not synchronise.  The first call on a device looks up the device address of
 * the scratch array (cudaGetSymbolAddress), so make that first call before any
 * stream capture; the address is kept for the life of the process and does not
 * survive cudaDeviceReset (do not call this entry point on a device after
 * resetting it).  All calls share the scratch array, which keeps the last
 * call's contents (each call overwrites what it reads); calls that overlap on
 * the GPU -- on different streams or from different threads -- race on it and
 * must be ordered by the caller.  Work per column is O(flops_j + min(flops_j,
 * m / 32)).  Returns SPGEMM_ERR_INVALID_ARG for a negative size or any null
 * array (Arowidx and Browidx included: with no nonzeros pass a one-element
 * array) and SPGEMM_ERR_CUDA when a CUDA call fails; an error already pending
 * from earlier work on the thread is cleared on entry, not reported. */
#define SPGEMM_NOALLOC_MAX_TILES 4096
#define SPGEMM_NOALLOC_MAX_ROWS 1048576
spgemm_status_t spgemm_colptr_noalloc(void* cuda_stream, int64_t m, int64_t k, int64_t n, const int64_t* Acolptr,
                                      const int32_t* Arowidx, const int64_t* Bcolptr, const int32_t* Browidx,
                                      int64_t* Ccolptr);

/* ---------------------------------------------------------------- learned predictor */
/* The nnz predictor is a small MLP (8 -> 32 -> 32 -> 1, ReLU, fp32) over per-column
 * features; it has no counterpart in the paper (its Section 8 lists structure
 * prediction as future work).  Parameters are held by the context. */
#define SPGEMM_PREDICTOR_NPARAM 1377
/* Copy NPARAM floats (host pointer) into the context's predictor. */
spgemm_status_t spgemm_predictor_set(spgemm_ctx_t ctx, const float* params_host);
spgemm_status_t spgemm_predictor_get(spgemm_ctx_t ctx, float* params_host);
/* Per-column features of C = A*B (device output, n x 8 floats row-major) and,
 * when nnz_out is non-NULL, the exact nnz per column from the symbolic pass
 * (device, n int64) -- the training labels. */
spgemm_status_t spgemm_predictor_features(spgemm_ctx_t ctx, spgemm_mat_t A, spgemm_mat_t B, float* features_dev,
                                          int64_t* nnz_out_dev);
/* One Adam step of the MSE loss on log1p(nnz) over a device batch
 * (X: N x 8 floats, y: N floats = log1p(nnz)); writes the loss (host) and,
 * if grad_host is non-NULL, the gradient before the step (host, NPARAM). */
spgemm_status_t spgemm_predictor_train_step(spgemm_ctx_t ctx, const float* X_dev, const float* y_dev, int64_t N,
                                            float lr, float* loss_host, float* grad_host);
/* Forward pass: pred_dev[i] = network(X[i]) (log1p scale). */
spgemm_status_t spgemm_predictor_forward(spgemm_ctx_t ctx, const float* X_dev, int64_t N, float* pred_dev);

#ifdef __cplusplus
}
#endif
#endif /* SPGEMM_H */
