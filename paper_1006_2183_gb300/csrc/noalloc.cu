// Column pointers of C = A*B without any device allocation.
//
// The regular symbolic pass (spgemm_symbolic) allocates its temporaries --
// per-column counts, bins, scan partial sums -- through the context allocator.
// Some callers cannot allocate device memory at the point where they need C's
// structure: applications that hand the library a fixed, pre-planned memory
// budget and must not grow it, code running on a latency-critical path where an
// allocation call (and the device synchronisation it may cause) is not
// acceptable, or plugins living inside a host program whose memory manager owns
// all device memory.  spgemm_colptr_noalloc serves them: the caller passes the
// operands and the output array, and the only scratch is the file-scope device
// array below.
//
// Scratch: g_scan_partials, SPGEMM_NOALLOC_MAX_TILES int64 partial sums of the
// column-count scan (one per tile of NA_TILE columns), 32 KiB on every GPU that
// loads the library, held until the process exits.  Every call shares it and it
// keeps the previous call's contents; each call rewrites every entry it reads
// before reading it, so nothing needs clearing, but two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on it.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace {

constexpr int NA_BLOCK = 1024;
constexpr int NA_ITEMS = 4;
constexpr int NA_TILE = NA_BLOCK * NA_ITEMS;                   // columns per scan tile
constexpr int64_t NA_MAX_TILES = SPGEMM_NOALLOC_MAX_TILES;     // 4096 -> 16,777,216 columns
constexpr int64_t NA_MAX_ROWS = SPGEMM_NOALLOC_MAX_ROWS;       // bitmap of m bits in shared memory
constexpr int NA_COUNT_BLOCK = 256;

__device__ __align__(256) long long g_scan_partials[NA_MAX_TILES];

// Per-device address of g_scan_partials (host code cannot use the symbol itself).
std::mutex g_mu;
long long* g_ptr[64] = {nullptr};

// nnz(C(:,j)) = number of distinct rows over A(:,k), k in B(:,j): rows marked in
// a shared-memory bitmap of m bits (one CTA per column).  A column with fewer
// products than bitmap words counts the bits its own atomics set and clears only
// the words it touched, so it costs O(flops_j); a denser column counts and clears
// the whole bitmap, O(m / 32) <= O(flops_j).  The bitmap is cleared once at start.
__global__ void __launch_bounds__(NA_COUNT_BLOCK) k_count_bitmap(int64_t m, int64_t na, const int64_t* __restrict__ Acp,
                                                                 const int32_t* __restrict__ Air,
                                                                 const int64_t* __restrict__ Bcp,
                                                                 const int32_t* __restrict__ Bir, int64_t n,
                                                                 int64_t* __restrict__ cnt_out) {
    extern __shared__ __align__(16) uint32_t bm[];
    __shared__ unsigned long long s_tot, s_flops;
    const int nw = (int)((m + 31) >> 5);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = NA_COUNT_BLOCK / 32;
    for (int w = threadIdx.x; w < nw; w += NA_COUNT_BLOCK) bm[w] = 0u;
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        if (threadIdx.x == 0) s_tot = s_flops = 0;
        __syncthreads();
        const int64_t b0 = Bcp[j], b1 = Bcp[j + 1];
        unsigned long long f = 0;
        for (int64_t t = b0 + threadIdx.x; t < b1; t += NA_COUNT_BLOCK) {
            const int32_t k = Bir[t];
            if (k >= 0 && k < na) f += (unsigned long long)(Acp[k + 1] - Acp[k]);
        }
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        if (lane == 0 && f) atomicAdd(&s_flops, f);
        __syncthreads();
        const bool sparse = s_flops < (unsigned long long)nw;
        unsigned long long c = 0;
        // one warp per entry of B(:,j), lanes walk A(:,k)
        for (int64_t t = b0 + warp; t < b1; t += nwarp) {
            const int32_t k = Bir[t];
            if (k < 0 || k >= na) continue;
            for (int64_t q = Acp[k] + lane; q < Acp[k + 1]; q += 32) {
                const int32_t r = Air[q];
                if (r < 0 || r >= m) continue;
                const uint32_t bit = 1u << (r & 31);
                const uint32_t old = atomicOr(&bm[r >> 5], bit);
                c += (old & bit) == 0;   // a row seen for the first time in this column
            }
        }
        if (!sparse) c = 0;
        __syncthreads();
        if (sparse) {
            // clear exactly the words this column touched
            for (int64_t t = b0 + warp; t < b1; t += nwarp) {
                const int32_t k = Bir[t];
                if (k < 0 || k >= na) continue;
                for (int64_t q = Acp[k] + lane; q < Acp[k + 1]; q += 32) {
                    const int32_t r = Air[q];
                    if (r >= 0 && r < m) bm[r >> 5] = 0u;
                }
            }
        } else {
            for (int w = threadIdx.x; w < nw; w += NA_COUNT_BLOCK) {
                c += __popc(bm[w]);
                bm[w] = 0u;
            }
        }
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0 && c) atomicAdd(&s_tot, c);
        __syncthreads();
        if (threadIdx.x == 0) cnt_out[j] = (int64_t)s_tot;
    }
}

__device__ __forceinline__ long long na_block_scan(long long v, long long* ws, long long& total) {
    long long x = v;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        long long s = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    const long long add = w > 0 ? ws[w - 1] : 0;
    total = ws[31];
    __syncthreads();
    return x + add;   // inclusive
}

// tile sums of v[0, n) into part[tile]
__global__ void __launch_bounds__(NA_BLOCK) k_na_tile_sums(const int64_t* __restrict__ v, int64_t n,
                                                            long long* __restrict__ part) {
    __shared__ long long ws[32];
    const int64_t base = (int64_t)blockIdx.x * NA_TILE + threadIdx.x * NA_ITEMS;
    long long s = 0;
#pragma unroll
    for (int i = 0; i < NA_ITEMS; ++i)
        if (base + i < n) s += v[base + i];
    long long total;
    na_block_scan(s, ws, total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// exclusive scan of the tile sums, one CTA
__global__ void __launch_bounds__(NA_BLOCK) k_na_scan_partials(long long* part, int64_t ntiles) {
    __shared__ long long ws[32];
    long long carry = 0;
    for (int64_t b0 = 0; b0 < ntiles; b0 += NA_BLOCK) {
        const int64_t i = b0 + threadIdx.x;
        const long long v = i < ntiles ? part[i] : 0;
        long long total;
        const long long inc = na_block_scan(v, ws, total);
        if (i < ntiles) part[i] = carry + inc - v;
        carry += total;
    }
}

// in place: v[i] <- sum_{t <= i} v[t] (each tile rewrites only its own entries)
__global__ void __launch_bounds__(NA_BLOCK) k_na_inclusive_apply(int64_t* __restrict__ v, int64_t n,
                                                                  const long long* __restrict__ part) {
    __shared__ long long ws[32];
    const int64_t base = (int64_t)blockIdx.x * NA_TILE + threadIdx.x * NA_ITEMS;
    long long x[NA_ITEMS];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < NA_ITEMS; ++i) {
        x[i] = base + i < n ? v[base + i] : 0;
        s += x[i];
    }
    long long total;
    long long run = na_block_scan(s, ws, total) - s + part[blockIdx.x];
#pragma unroll
    for (int i = 0; i < NA_ITEMS; ++i) {
        run += x[i];
        if (base + i < n) v[base + i] = run;
    }
}

}  // namespace

extern "C" spgemm_status_t spgemm_colptr_noalloc(void* cuda_stream, int64_t m, int64_t k, int64_t n,
                                                 const int64_t* Acolptr, const int32_t* Arowidx,
                                                 const int64_t* Bcolptr, const int32_t* Browidx, int64_t* Ccolptr) {
    // every array must be a real device pointer: a caller with no nonzeros still passes
    // a one-element row array
    if (m < 0 || k < 0 || n < 0 || !Acolptr || !Arowidx || !Bcolptr || !Browidx || !Ccolptr)
        return SPGEMM_ERR_INVALID_ARG;
    if (m > NA_MAX_ROWS) return SPGEMM_ERR_UNSUPPORTED;                        // bitmap must fit shared memory
    if (sg::ceil_div64(std::max<int64_t>(n, 1), NA_TILE) > NA_MAX_TILES) return SPGEMM_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SPGEMM_ERR_CUDA;
    long long* part = nullptr;
    {
        // first call on this device: look up the device address of the scratch array
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scan_partials) != cudaSuccess) {
                cudaGetLastError();
                return SPGEMM_ERR_CUDA;
            }
            g_ptr[dev] = (long long*)p;
        }
        part = g_ptr[dev];
    }
    // an error left pending by earlier, unrelated work would otherwise be reported
    // as this call's failure by the check after the launches; a sticky error
    // (a lost context) is reported by the first call below
    cudaGetLastError();
    if (cudaMemsetAsync(Ccolptr, 0, sizeof(int64_t), st) != cudaSuccess) return SPGEMM_ERR_CUDA;
    if (n == 0) return SPGEMM_OK;
    int64_t* cnt = Ccolptr + 1;   // counts land in Ccolptr[1..n], then are scanned in place
    const size_t smem = (size_t)((m + 31) / 32) * 4;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_count_bitmap, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SPGEMM_ERR_CUDA;
    const int grid = (int)std::min<int64_t>(n, sg::sm_count() * 8);
    k_count_bitmap<<<grid, NA_COUNT_BLOCK, smem, st>>>(m, k, Acolptr, Arowidx, Bcolptr, Browidx, n, cnt);
    const int64_t ntiles = sg::ceil_div64(n, NA_TILE);
    k_na_tile_sums<<<(int)ntiles, NA_BLOCK, 0, st>>>(cnt, n, part);
    k_na_scan_partials<<<1, NA_BLOCK, 0, st>>>(part, ntiles);
    k_na_inclusive_apply<<<(int)ntiles, NA_BLOCK, 0, st>>>(cnt, n, part);
    sg::note_launch(4);
    return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}
