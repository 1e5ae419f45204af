// Kernel launch interface of the flat SpGEMM path (host side of kernels.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace sg {

// Column tiers.  A column's capacity bound is cap_j = min(flops_j, m) >= nnz(C(:,j)).
//   bin 0                  : cap == 0 (empty output column)
//   bins 1 .. NWARP        : warp-wide hash tables of 64 .. 1024 slots (>= 2 cap)
//   bins NWARP+1 .. +NBLK  : CTA-wide hash tables of 2048 .. 8192 slots (>= 2 cap)
//   bin NBIN-1             : row-chunked dense accumulator, column split into parts
constexpr int NWARP = 5;
constexpr int NBLK = 3;
constexpr int NBIN = 1 + NWARP + NBLK + 1;
constexpr int BIN_DENSE = NBIN - 1;
constexpr int WARP_TBL0 = 64;
constexpr int BLK_TBL0 = 2048;
constexpr int MAX_PARTS = 16;

struct TierCfg {
    int warp_max;     // cap <= warp_max -> warp tables (<= 512)
    int block_max;    // cap <= block_max -> CTA tables (<= 4096)
    int dense_rows;   // R, rows per dense chunk
    int part_flops;   // target flops per dense part
};

struct FeatOut {          // optional per-column predictor inputs
    float* x = nullptr;   // n x 8, row-major
};

// which: 1 = hash-table tiers, 2 = dense tier, 3 = both
// per stored column p of B: flops, tier bin; bin counts accumulated into bin_count[NBIN].
void launch_analyze(cudaStream_t st, const DMat& A, const DMat& B, TierCfg cfg, int64_t* flops, uint8_t* bin,
                    unsigned long long* bin_count, unsigned long long* flops_total, const uint64_t* sketch_A,
                    float* feat);
void launch_bin_scatter(cudaStream_t st, int64_t n, const uint8_t* bin, const int64_t* bin_off,
                        unsigned long long* bin_cursor, int32_t* list);
// dense items: (list position d, part q) for each dense column
void launch_dense_items(cudaStream_t st, const int32_t* dense_list, int64_t ndense, const int64_t* flops,
                        int G, int part_flops, int2* items, unsigned long long* nitems, int8_t* nparts);
void launch_row_sketch(cudaStream_t st, const DMat& A, uint64_t* sketch);

template <class SR>
void launch_symbolic(cudaStream_t st, const DMat& A, const DMat& B, TierCfg cfg, const int32_t* list,
                     const int64_t* bin_off, const int64_t* bin_cnt, const int2* dense_items,
                     const unsigned long long* nitems, int64_t nitems_host, const int8_t* nparts, int32_t* cursors,
                     int32_t* part_count, int64_t* nnz_col, int which = 3);
template <class SR>
void launch_numeric(cudaStream_t st, const DMat& A, const DMat& B, TierCfg cfg, const int32_t* list,
                    const int64_t* bin_off, const int64_t* bin_cnt, const int2* dense_items,
                    const unsigned long long* nitems, int64_t nitems_host, int32_t* cursors,
                    const int32_t* part_count, const int8_t* nparts, const int64_t* Ccp, int32_t* Cir,
                    typename SR::T* Cv, int which = 3);

// nnz of dense columns = sum of their part counts
void launch_sum_parts(cudaStream_t st, const int32_t* dense_list, int64_t ndense, const int8_t* nparts,
                      const int32_t* part_count, int64_t* nnz_col, const int32_t* jc);
// out[0] = 0, out[i+1] = sum_{t <= i} in[t]; tmp needs scan_tmp_bytes(n)
size_t scan_tmp_bytes(int64_t n);
void launch_exclusive_scan(cudaStream_t st, const int64_t* in, int64_t n, int64_t* out, void* tmp);
void launch_fill_i64(cudaStream_t st, int64_t* p, int64_t n, int64_t v);

int dense_rows_for(int semiring, int requested);

// process-wide count of kernel launches made by this library
void note_launch(int n = 1);
int64_t launches();

// per-tier totals {cols, flops, nnz(C), nnz(B)} x 4 tiers into out[16] (device, zeroed by caller)
void launch_tier_stats(cudaStream_t st, const uint8_t* bin, const int64_t* flops, const int64_t* nnz_col,
                       const int32_t* jc, const int64_t* bcp, int64_t nzc, unsigned long long* out);

}  // namespace sg
