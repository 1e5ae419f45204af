// Kernel launch interface of the batched column-wise SpGEMM (host side of kernels.cu).
//
// Work is expressed in an "item space": a batch holds nprod products
// C_i = A_i * B_i (descriptors in device memory); item u = item_base_i + p is the
// p-th stored column of B_i and produces one output column (or one DCSC column).
// The flat product is a batch of one; the SUMMA stage products, the stage merge
// and spgemm_batch are larger batches.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace sg {

// Column tiers.  An item's capacity bound is cap = min(flops, m) >= nnz of its output.
//   bin 0                  : cap == 0 (empty output column)
//   bin 1                  : flops <= TINY_MAX: one thread, products sorted in registers
//   bins 2 .. NWARP+1      : warp-wide hash tables of 64 .. 1024 slots (>= 2 cap)
//   bins NWARP+2 .. +NBLK  : CTA-wide hash tables of 2048 .. 8192 slots (>= 2 cap)
//   bin NBIN-1             : slab tier (long columns cut into row slabs)
constexpr int NWARP = 5;
constexpr int NBLK = 3;
constexpr int NBIN = 2 + NWARP + NBLK + 1;
constexpr int BIN_TINY = 1;
constexpr int BIN_WARP0 = 2;
constexpr int BIN_BLK0 = BIN_WARP0 + NWARP;
constexpr int BIN_DENSE = NBIN - 1;
constexpr int TINY_MAX = 16;
constexpr int WARP_TBL0 = 64;
constexpr int BLK_TBL0 = 2048;
// most row slabs of one long column
constexpr int MAX_PARTS = 64;
// default most rows of one slab: a 64 KB row bitmap keeps two CTAs per SM
constexpr int DEFAULT_SLAB_ROWS = 1 << 19;
// default target flops per slab: every slab repeats its binary searches per entry of
// B(:,j) and its bitmap set-up, so larger slabs pay up to about this size (R-MAT
// scale 20 flat: 8192 / 16384 / 32768 / 65536 / 131072 flops per slab give 74.8 /
// 67.9 / 64.5 / 62.3 / 62.1 ms for the FP64 numeric pass)
constexpr int DEFAULT_PART_FLOPS = 65536;

struct TierCfg {
    int warp_max;     // cap <= warp_max -> warp tables (<= 512)
    int block_max;    // cap <= block_max -> CTA tables (<= 4096)
    int sort_max = 0; // > 0 (operands of at most BLOCK_TIER_MAX_ROWS rows): bins 2, 3 and 4
                      // hold only columns of at most 32, 64 and 128 products (the sort tier)
    int dense_rows;   // RB, most rows of one slab (bitmap bits in shared memory)
    int part_flops;   // target flops per slab of a long column
};

// Everything a pass needs about slab s before its work starts, written by the
// boundary pre-pass (and, for the numeric pass, completed once C's offsets are
// known): the passes copy the next slab's record into shared memory while the
// current slab runs, so a slab starts without a chain of dependent loads.
struct __align__(16) SlabRec {
    int32_t prod, col;   // the long column: product and stored column of B
    int32_t r0, r1;      // rows [r0, r1) of the slab
    int32_t rb;          // output row base of the column
    int32_t cnt;         // rows of the slab's row set (counting pass)
    int64_t bs, be;      // B(:,j) is entries [bs, be)
    int64_t bnd;         // this slab's row of the boundary table in `bnd`
    int64_t u;           // item index of the column
    int64_t ob;          // where the slab's rows start in C (numeric pass)
    int64_t soff;        // where its row set is stored (< 0: none)
    int64_t sab;         // the column's rows P + 1 and P + 2 of `bnd`: where each A(:,k) starts
};
static_assert(sizeof(SlabRec) == 80, "five 16-byte chunks");

// State of the slab tier shared by its kernels.  Slab s = sbase[d] + q is slab q
// of long column d (position d in the dense list); items[s] = (d, q).
struct DenseWork {
    const int2* dlist = nullptr;          // long columns (product, stored column)
    int64_t ndense = 0;
    const int2* items = nullptr;          // slabs (d, q)
    const unsigned long long* nitems = nullptr;   // device count of slabs
    int64_t nslabs = 0;                   // host copy of the count (0 before it is known)
    const int8_t* nparts = nullptr;       // slabs per long column
    const int32_t* sbase = nullptr;       // first slab of each long column
    int32_t* scount = nullptr;            // rows per slab (symbolic pass)
    int32_t* spref = nullptr;             // rows of the column's earlier slabs
    int64_t* soff = nullptr;              // where each slab's row set is stored
    uint32_t* store = nullptr;            // row sets: bitmap words, or rows ascending
    int64_t store_cap = 0;                // entries of store
    unsigned long long* store_ctr = nullptr;
    const int* vals_zero = nullptr;       // boolean semiring: some operand value is false
    int32_t* bnd = nullptr;               // slab boundaries: per long column, P + 3 rows of deg:
                                          // offsets into every A(:,k) (row P: its length),
                                          // then where A(:,k) starts (low, high 32 bits)
    const int64_t* bbase = nullptr;       // where each long column's boundary table starts
    SlabRec* rec = nullptr;               // per slab: its record
    int* err = nullptr;                   // nonzero: a capacity was exceeded
    int RB = 1 << 19;                     // most rows per slab
    // block mode (every A_i has at most BLOCK_TIER_MAX_ROWS rows): long columns
    // are counted with row bitmaps and computed by the block tier; no slabs
    bool dcol = false;
};

// Products whose every A_i has at most this many rows run their numeric pass in
// the block tier (two-level row bitmap per column, L2 reductions; blocktier.cu)
// and count their columns with row bitmaps.
constexpr int BLOCK_TIER_MAX_ROWS = 32768;

struct Items {
    const Prod* prods = nullptr;        // device, nprod descriptors
    const int64_t* item_base = nullptr; // device, nprod + 1 (prefix of stored columns of B_i)
    int64_t nprod = 0;
    int64_t nitems = 0;
    int64_t total_bnz = 0;              // sum of nnz(B_i): cursor stride per dense part
    int64_t max_m = 0;                  // most rows of any A_i
    // A-column cache (DCSC A only): for every stored entry B_i(k, j), where A_i(:,k)
    // starts and how long it is, filled by the analysis pass so that later passes
    // skip the DCSC lookup.  Indexed by bnz_base + position within B_i.
    int64_t* acs = nullptr;
    int32_t* acl = nullptr;
};

// A(:,k) for the B entry at position t of product pr (cached when the engine has
// the A-column cache, else looked up).
__device__ __forceinline__ void a_col(const Items& it, const Prod* pr, int64_t t, int32_t k, int64_t& s, int64_t& e) {
    if (it.acs) {
        const int64_t i = pr->bnz_base + (t - __ldg(pr->B.cp));
        s = __ldg(it.acs + i);
        e = s + __ldg(it.acl + i);
    } else {
        col_range(pr->A, k, s, e);
    }
}

// CTA-wide hash tables order their numeric output through a shared-memory row
// bitmap (instead of sorting) when every A_i has at most this many rows.
constexpr int64_t BM_MAX_ROWS = 262144;
// The same for warp tables (one bitmap per warp), and only where sorting costs more.
constexpr int64_t BM_WARP_MAX_ROWS = 32768;
constexpr int BM_WARP_MIN_TBL = 256;   // smaller tables hold too few rows to prefer the bitmap

// flops and bin per item, product id per item, bin counts and total flops.
// With feat != nullptr also the 8 predictor inputs per item; `sketch` holds the
// per-column row sketches of the A operands concatenated, product i's starting
// at sketch_base[i].
void launch_analyze(cudaStream_t st, const Items& it, TierCfg cfg, int64_t* flops, uint8_t* bin, int32_t* item_prod,
                    unsigned long long* bin_count, unsigned long long* flops_total, const uint64_t* sketch,
                    const int64_t* sketch_base, float* feat, int64_t* maxlen = nullptr);
void launch_row_sketch(cudaStream_t st, const DMat& A, uint64_t* sketch);
void launch_bin_scatter(cudaStream_t st, const Items& it, const uint8_t* bin, const int32_t* item_prod,
                        const int64_t* bin_off, unsigned long long* bin_cursor, int2* list);
// hash-tier bins from exact counts (after the symbolic pass); cnt[NBIN] accumulates
void launch_numeric_bins(cudaStream_t st, const Items& it, TierCfg cfg, const uint8_t* bin, const int64_t* flops,
                         const int64_t* nnz_item, uint8_t* nbin, unsigned long long* cnt);
// slabs of the long columns (position d in the dense list, slab q); P_d slabs of at
// most RB rows each; *store_bound accumulates the entries their row sets can need
void launch_dense_items(cudaStream_t st, const Items& it, const int2* dense_list, int64_t ndense,
                        const int64_t* flops, int part_flops, int RB, int2* items, unsigned long long* nitems,
                        int8_t* nparts, int32_t* sbase, unsigned long long* store_bound, int64_t* bbase,
                        unsigned long long* bnd_total);
// *flag = 1 when an operand of some product stores a false value (boolean semiring)
void launch_false_values(cudaStream_t st, const Items& it, int* flag);
// *flag = 1 when one of the n bytes at vals is 0 (vals == nullptr: nothing)
void launch_any_false(cudaStream_t st, const void* vals, int64_t n, int* flag);

// which: 1 = hash-table tiers, 2 = long columns (slab tier, or the block tier in block mode), 3 = both
template <class SR>
void launch_symbolic(cudaStream_t st, const Items& it, TierCfg cfg, const int2* list, const int64_t* bin_off,
                     const int64_t* bin_cnt, const DenseWork& dw, int64_t* nnz_item, int which = 3);
template <class SR>
void launch_numeric(cudaStream_t st, const Items& it, TierCfg cfg, const int2* list, const int64_t* bin_off,
                    const int64_t* bin_cnt, const DenseWork& dw, const int64_t* Coff, int32_t* Cir,
                    typename SR::T* Cv, int which = 3);

// numeric pass of the hash tiers into a predicted layout: cap_off are capacity offsets;
// every item's exact count goes to nnz_item, items that do not fit are not written
template <class SR>
void launch_numeric_predicted(cudaStream_t st, const Items& it, const int2* list, const int64_t* bin_off,
                              const int64_t* bin_cnt, const DenseWork& dw, const int64_t* cap_off, int64_t* nnz_item,
                              int32_t* Cir, typename SR::T* Cv);

// numeric pass of the block tier (blocktier.cu); with nnz_item the counts are recorded and
// a column is written only when it fits its slots Coff[u+1] - Coff[u]
template <class SR>
void launch_block_tier(cudaStream_t st, const Items& it, const int2* list, const int64_t* bin_off,
                       const int64_t* bin_cnt, const DenseWork& dw, int64_t* nnz_item, const int64_t* Coff,
                       int32_t* Cir, typename SR::T* Cv, int which);
// nnz of long columns = sum of their slab counts (and each slab's start in its column)
void launch_sum_parts(cudaStream_t st, const Items& it, const DenseWork& dw, int64_t* nnz_item);
// per-product column pointers from item offsets: out[colbase_i + j] for j in [0, n_i]
void launch_colptrs(cudaStream_t st, const Items& it, const int64_t* colbase, int64_t total_cols, const int64_t* Coff,
                    int64_t* out);
// out[i] = Coff[item_base[i]] for i in [0, np]: where each product's output starts
void launch_gather_offsets(cudaStream_t st, const int64_t* Coff, const int64_t* item_base, int64_t np, int64_t* out);
// out[0] = 0, out[i+1] = sum_{t <= i} in[t]; tmp needs scan_tmp_bytes(n)
size_t scan_tmp_bytes(int64_t n);
void launch_exclusive_scan(cudaStream_t st, const int64_t* in, int64_t n, int64_t* out, void* tmp);
void launch_fill_i64(cudaStream_t st, int64_t* p, int64_t n, int64_t v);
// per-tier totals {cols, flops, nnz(C), nnz(B)} x 4 tiers into out[16] (device, zeroed by caller)
void launch_tier_stats(cudaStream_t st, const Items& it, const uint8_t* bin, const int32_t* item_prod,
                       const int64_t* flops, const int64_t* nnz_item, unsigned long long* out);


// streaming multiprocessors of the current device (queried once per device)
int sm_count();

// process-wide count of kernel launches made by this library
void note_launch(int n = 1);
int64_t launches();

}  // namespace sg
