// Batched column-wise SpGEMM kernels (Gustavson's column-by-column
// formulation, Section 2.1; accumulation in the spirit of the sparse
// accumulator of Section 3.3), organised in accumulator tiers chosen per
// output column from cap = min(flops, m):
//   * one thread per column for flops <= 16 (insertion sort in registers),
//   * warp-wide shared-memory hash tables (short columns),
//   * CTA-wide shared-memory hash tables (medium columns),
//   * the range tier (long columns): the symbolic pass marks the column's rows
//     in a shared-memory bitmap per row slab and cuts the slab into row ranges
//     of bounded output; the numeric pass walks the ranges in row order with
//     per-(column, k) cursors into A(:,k), accumulates each range in a hash
//     table (or a dense row array when the range is narrow) and writes it out
//     in row order through the range's bitmap.
// The symbolic pass counts nnz per output column; the numeric pass fills rows
// and values, in ascending row order without a sort wherever a row bitmap fits
// in shared memory.  Every kernel works on items (product, stored column of B).
#include <algorithm>
#include <atomic>
#include <climits>
#include <map>
#include <mutex>
#include <utility>

#include "kernels.cuh"

namespace sg {

static std::atomic<int64_t> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches() { return g_launches.load(std::memory_order_relaxed); }

int sm_count() {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto f = cache.find(dev);
    if (f != cache.end()) return f->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return 1;   // not cached: asked again next time
    }
    cache[dev] = n;
    return n;
}

// Raises a kernel's dynamic shared-memory limit on the current device to at least
// `bytes`; never lowers it (the limit belongs to the kernel, whichever launcher
// asks).  A refused request is not remembered, so the launch reports the error.
static void smem_at_least(const void* fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> limit;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    size_t& cur = limit[{dev, fn}];
    if (cur < bytes && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess)
        cur = bytes;
}

constexpr int WARP_BLOCK = 256;   // 8 warp groups per CTA

__host__ __device__ __forceinline__ int bin_of(int64_t flops, int64_t cap, int warp_max, int block_max,
                                              int sort_max) {
    if (cap <= 0) return 0;
    if (flops <= TINY_MAX) return BIN_TINY;
    if (cap <= warp_max) {
        // with sort_max, a column of more than sort_max products never lands in a bin
        // whose table is for at most sort_max rows: bins 2 and 3 then also bound flops
        int64_t c = cap;
        if (sort_max > 0) {
            const int64_t fl = flops < sort_max + 1 ? flops : sort_max + 1;
            c = cap > fl ? cap : fl;
        }
        int64_t t = WARP_TBL0;
        int b = BIN_WARP0;
        while (t < 2 * c) { t <<= 1; ++b; }
        return b;
    }
    if (cap <= block_max) {
        int64_t t = BLK_TBL0;
        int b = BIN_BLK0;
        while (t < 2 * cap) { t <<= 1; ++b; }
        return b;
    }
    return BIN_DENSE;
}

__device__ __forceinline__ int find_prod(const int64_t* __restrict__ base, int64_t nprod, int64_t u) {
    // last product i with base[i] <= u
    int64_t lo = 0, hi = nprod - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= u) lo = mid;
        else hi = mid - 1;
    }
    return (int)lo;
}

__device__ __forceinline__ int64_t out_col(const DMat& B, int64_t p) { return B.jc ? __ldg(B.jc + p) : p; }

// ------------------------------------------------------------------ analysis
// Groups of LPI lanes per item (8, or 1 where B columns are short, as in the
// block products): flops = sum_k nnz(A(:,k)) (Section 1's flops), the tier bin,
// the product id, and optionally the predictor inputs.
template <int LPI>
__global__ void __launch_bounds__(256) k_analyze(Items it, TierCfg cfg, int64_t* __restrict__ flops,
                                                 uint8_t* __restrict__ bin, int32_t* __restrict__ item_prod,
                                                 unsigned long long* bin_count, unsigned long long* flops_total,
                                                 const uint64_t* __restrict__ sketch,
                                                 const int64_t* __restrict__ sketch_base, float* __restrict__ feat,
                                                 int64_t* __restrict__ maxlen) {
    __shared__ unsigned long long s_cnt[NBIN];
    __shared__ unsigned long long s_fl;
    if (threadIdx.x < NBIN) s_cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_fl = 0;
    __syncthreads();
    const int sub = threadIdx.x & (LPI - 1);
    const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / LPI;
    long long f = 0, mx = 0;
    unsigned long long sk = 0;
    int64_t bs = 0, be = 0, am = 0;
    int prod = 0;
    if (u < it.nitems) {
        prod = it.nprod == 1 ? 0 : __ldg(item_prod + u);   // filled per product beforehand
        const Prod* pr = it.prods + prod;
        const int64_t p = u - __ldg(it.item_base + prod);
        bs = __ldg(pr->B.cp + p);
        be = __ldg(pr->B.cp + p + 1);
        am = pr->A.m;
        const uint64_t* skp = sketch ? sketch + sketch_base[prod] : nullptr;
        const int64_t b0 = it.acs ? pr->bnz_base - __ldg(pr->B.cp) : 0;
        if constexpr (LPI == 1) {
            // two entries of B(:,j) at a time, each step of their A-column lookups issued
            // for both before either is used (a lookup is a chain of dependent loads: B's
            // row, then AUX, then JC, then CP)
            const DMat& A = pr->A;
            for (int64_t t0 = bs; t0 < be; t0 += 2) {
                int32_t k[2];
#pragma unroll
                for (int i = 0; i < 2; ++i) k[i] = t0 + i < be ? __ldg(pr->B.ir + t0 + i) : -1;
                int64_t cs[2], ce[2];
                col_range2(A, k, cs, ce);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    if (t0 + i >= be) break;
                    const long long len = ce[i] - cs[i];
                    if (it.acs) {   // fill the A-column cache for the later passes
                        it.acs[b0 + t0 + i] = cs[i];
                        it.acl[b0 + t0 + i] = (int32_t)len;
                    }
                    f += len;
                    mx = len > mx ? len : mx;
                    if (skp && k[i] >= 0 && k[i] < A.n) sk |= __ldg(skp + k[i]);
                }
            }
        } else {
            for (int64_t t = bs + sub; t < be; t += LPI) {
                int32_t k = __ldg(pr->B.ir + t);
                int64_t cs, ce;
                col_range(pr->A, k, cs, ce);
                long long len = ce - cs;
                if (it.acs) {   // fill the A-column cache for the later passes
                    it.acs[b0 + t] = cs;
                    it.acl[b0 + t] = (int32_t)len;
                }
                f += len;
                mx = len > mx ? len : mx;
                if (skp && k >= 0 && k < pr->A.n) sk |= __ldg(skp + k);
            }
        }
    }
#pragma unroll
    for (int o = LPI / 2; o > 0; o >>= 1) {
        f += __shfl_xor_sync(0xffffffffu, f, o, LPI);
        long long om = __shfl_xor_sync(0xffffffffu, mx, o, LPI);
        mx = om > mx ? om : mx;
        sk |= __shfl_xor_sync(0xffffffffu, sk, o, LPI);
    }
    const bool has = u < it.nitems && sub == 0;
    const int64_t cap = f < am ? f : am;
    const int b = has ? bin_of(f, cap, cfg.warp_max, cfg.block_max, cfg.sort_max) : -1;
    {
        // per-bin counts and total flops, one shared atomic per bin per warp (every
        // item of a CTA adding to the same few counters serialises on them)
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int lane = threadIdx.x & 31;
        if (has && lane == __ffs(peers) - 1) atomicAdd(&s_cnt[b], (unsigned long long)__popc(peers));
        unsigned long long fs = has ? (unsigned long long)f : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fs += __shfl_xor_sync(0xffffffffu, fs, o);
        if (lane == 0 && fs) atomicAdd(&s_fl, fs);
    }
    if (has) {
        flops[u] = f;
        if (it.nprod == 1) item_prod[u] = 0;
        bin[u] = (uint8_t)b;
        if (maxlen) maxlen[u] = mx;
        if (feat) {
            // predictor inputs (definitions in predictor.cu)
            float d = (float)(be - bs);
            int pc = __popcll(sk);
            float pcf = fminf((float)pc, 63.5f);
            float lc = 64.0f * logf(64.0f / (64.0f - pcf));
            float* x = feat + u * 8;
            x[0] = log1pf(d);
            x[1] = log1pf((float)f);
            x[2] = log1pf((float)mx);
            x[3] = log1pf((float)am);
            x[4] = log1pf(lc);
            x[5] = log1pf((float)cap);
            x[6] = log1pf((float)(f - mx));
            x[7] = (float)pc * (1.0f / 64.0f);
        }
    }
    __syncthreads();
    if (threadIdx.x < NBIN && s_cnt[threadIdx.x]) atomicAdd(bin_count + threadIdx.x, s_cnt[threadIdx.x]);
    if (threadIdx.x == 0 && flops_total) atomicAdd(flops_total, s_fl);
}

// item_prod[u] = the product of item u: one CTA per product over its contiguous items.
__global__ void k_item_prod(Items it, int32_t* __restrict__ item_prod) {
    const int64_t p = blockIdx.x;
    const int64_t u0 = __ldg(it.item_base + p), u1 = __ldg(it.item_base + p + 1);
    for (int64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) item_prod[u] = (int32_t)p;
}

void launch_analyze(cudaStream_t st, const Items& it, TierCfg cfg, int64_t* flops, uint8_t* bin, int32_t* item_prod,
                    unsigned long long* bin_count, unsigned long long* flops_total, const uint64_t* sketch,
                    const int64_t* sketch_base, float* feat, int64_t* maxlen) {
    if (it.nitems == 0) return;
    if (it.nprod > 1) {
        k_item_prod<<<(unsigned)it.nprod, 256, 0, st>>>(it, item_prod);
        note_launch();
    }
    if (it.total_bnz < 4 * it.nitems) {   // about one B entry per item: one lane each
        int grid = (int)ceil_div64(it.nitems, 256);
        k_analyze<1><<<grid, 256, 0, st>>>(it, cfg, flops, bin, item_prod, bin_count, flops_total, sketch,
                                           sketch_base, feat, maxlen);
    } else {
        int grid = (int)ceil_div64(it.nitems * 8, 256);
        k_analyze<8><<<grid, 256, 0, st>>>(it, cfg, flops, bin, item_prod, bin_count, flops_total, sketch,
                                           sketch_base, feat, maxlen);
    }
    note_launch();
}

// sketch(A(:,k)) = OR over rows i of 2^(bits 31..26 of i * 0x9E3779B1)
__global__ void k_row_sketch(DMat A, uint64_t* __restrict__ sk) {
    int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    int sub = threadIdx.x & 7;
    unsigned long long v = 0;
    if (p < A.nzc) {
        int64_t s = __ldg(A.cp + p), e = A.ce ? __ldg(A.ce + p) : __ldg(A.cp + p + 1);
        for (int64_t t = s + sub; t < e; t += 8) {
            uint32_t h = (uint32_t)__ldg(A.ir + t) * 0x9E3779B1u;
            v |= 1ull << (h >> 26);
        }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o, 8);
    if (p < A.nzc && sub == 0) sk[A.jc ? __ldg(A.jc + p) : p] = v;
}

void launch_row_sketch(cudaStream_t st, const DMat& A, uint64_t* sketch) {
    if (A.jc) cudaMemsetAsync(sketch, 0, sizeof(uint64_t) * std::max<int64_t>(A.n, 1), st);
    if (A.nzc == 0) return;
    k_row_sketch<<<(int)ceil_div64(A.nzc * 8, 256), 256, 0, st>>>(A, sketch);
    note_launch();
}

// Numeric bins of the hash-tier items from their exact counts: the table needs
// only 2 nnz slots, not 2 min(flops, m).  Range-tier and empty items get bin 0
// (not listed).
__global__ void k_numeric_bins(Items it, TierCfg cfg, const uint8_t* __restrict__ bin,
                               const int64_t* __restrict__ flops, const int64_t* __restrict__ nnz_item,
                               uint8_t* __restrict__ nbin, unsigned long long* __restrict__ cnt) {
    __shared__ unsigned long long s_cnt[NBIN];
    for (int b = threadIdx.x; b < NBIN; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < it.nitems; u += (int64_t)gridDim.x * blockDim.x) {
        const int b = bin[u];
        int nb = 0;
        if (b >= BIN_TINY && b < BIN_DENSE) nb = bin_of(flops[u], nnz_item[u], cfg.warp_max, cfg.block_max, cfg.sort_max);
        nbin[u] = (uint8_t)nb;
        if (nb) atomicAdd(&s_cnt[nb], 1ull);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < NBIN; b += blockDim.x)
        if (s_cnt[b]) atomicAdd(cnt + b, s_cnt[b]);
}

void launch_numeric_bins(cudaStream_t st, const Items& it, TierCfg cfg, const uint8_t* bin, const int64_t* flops,
                         const int64_t* nnz_item, uint8_t* nbin, unsigned long long* cnt) {
    if (it.nitems == 0) return;
    const int grid = (int)std::min<int64_t>(ceil_div64(it.nitems, 256), sm_count() * 8);
    k_numeric_bins<<<grid, 256, 0, st>>>(it, cfg, bin, flops, nnz_item, nbin, cnt);
    note_launch();
}

// Scatter of items into per-bin lists (warp-aggregated atomics).
__global__ void k_bin_scatter(Items it, const uint8_t* __restrict__ bin, const int32_t* __restrict__ item_prod,
                              const int64_t* __restrict__ bin_off, unsigned long long* cursor, int2* __restrict__ list) {
    int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int b = u < it.nitems ? bin[u] : -1;
    unsigned mask = __match_any_sync(0xffffffffu, b);
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (b > 0 && lane == leader) base = atomicAdd(cursor + b, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (b > 0) {
        int rank = __popc(mask & ((1u << lane) - 1));
        int prod = item_prod[u];
        int p = (int)(u - __ldg(it.item_base + prod));
        list[bin_off[b] + base + rank] = make_int2(prod, p);
    }
}

void launch_bin_scatter(cudaStream_t st, const Items& it, const uint8_t* bin, const int32_t* item_prod,
                        const int64_t* bin_off, unsigned long long* bin_cursor, int2* list) {
    if (it.nitems == 0) return;
    k_bin_scatter<<<(int)ceil_div64(it.nitems, 256), 256, 0, st>>>(it, bin, item_prod, bin_off, bin_cursor, list);
    note_launch();
}

// ------------------------------------------------------------------ hash tiers
template <class SR, int GS, int TBL, bool NUM>
struct HashLayout {
    using T = typename SR::T;
    using Acc = typename SR::Acc;
    static constexpr size_t keys = (size_t)TBL * 4;
    static constexpr size_t vals = NUM ? (size_t)TBL * sizeof(Acc) : 0;
    static constexpr size_t incl = (size_t)GS * 4;
    static constexpr size_t a0 = (size_t)GS * 8;
    static constexpr size_t bv = NUM ? (size_t)GS * 8 : 0;
    static constexpr size_t scan = 33 * 4 + 4;
    static constexpr size_t group = (keys + vals + incl + a0 + bv + scan + 15) / 16 * 16;
};

template <int GS, class Acc>
__device__ __forceinline__ void bitonic_sort(int32_t* keys, Acc* vals, int P) {
    using G = Group<GS>;
    const int lane = G::lane();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = lane; t < (P >> 1); t += GS) {
                int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                int l = i + j;
                bool asc = (i & k) == 0;
                int32_t ki = keys[i], kl = keys[l];
                if ((ki > kl) == asc) {
                    keys[i] = kl;
                    keys[l] = ki;
                    Acc vi = vals[i];
                    vals[i] = vals[l];
                    vals[l] = vi;
                }
            }
            G::sync();
        }
    }
}

// Writes a group's table in row order: the rank of row r among the marked rows of
// `bitmap` (nw words) is the number of bits below it, from per-member prefix counts
// of groups of gw words plus the popcounts inside r's group, so every occupied slot
// writes its entry at its rank directly (no sort, no probing).  Empties the table
// and the bitmap.  Called by all GS members; returns the number of entries.  With
// `pred`, nothing is written when the count exceeds capn.
template <class SR, int TBL, int GS>
__device__ __forceinline__ int rank_emit(uint32_t* bitmap, uint16_t* wp, int nw, int32_t* keys,
                                         typename SR::Acc* vals, int* gp, int* scratch, bool pred, int64_t capn,
                                         int64_t out0, int32_t rb, int32_t* __restrict__ Cir,
                                         typename SR::T* __restrict__ Cv) {
    using G = Group<GS>;
    const int lane = G::lane();
    int lgw = 0;   // words per member: a power of two with GS members covering nw words
    while ((GS << lgw) < nw) ++lgw;
    const int gw = 1 << lgw;
    // wp[x]: set bits before word x within its member's words (< 2^16: gw <= 2^11)
    int c = 0;
    for (int x = lane * gw; x < (lane + 1) * gw && x < nw; ++x) {
        wp[x] = (uint16_t)c;
        c += __popc(bitmap[x]);
    }
    int total;
    const int incl = group_incl_scan<GS>(c, scratch, total);
    gp[lane] = incl - c;
    G::sync();
    const bool write = !pred || total <= capn;
    for (int s = lane; s < TBL; s += GS) {
        const int32_t kr = keys[s];
        if (kr < 0) continue;
        const int wd = kr >> 5;
        if (wd < nw && write) {   // rows past the bitmap occur only on malformed input
            const int rank = gp[wd >> lgw] + wp[wd] + __popc(bitmap[wd] & ((1u << (kr & 31)) - 1u));
            Cir[out0 + rank] = kr + rb;
            Cv[out0 + rank] = SR::out(vals[s]);
        }
        keys[s] = -1;
        vals[s] = SR::zero();
    }
    G::sync();
    for (int x = lane; x < nw; x += GS) bitmap[x] = 0u;
    G::sync();
    return total;
}

// The hash tables are latency-bound: registers are capped so that they never admit
// fewer CTAs per SM than shared memory does (48 warps for warp tables, tables of 2
// or 4 warps and 2048-slot CTA tables; 4 CTAs of 4096 slots; 2 CTAs of 512 threads).
constexpr int hash_min_blocks(int block, int tbl) {
    return block <= 128 ? 1536 / block : block == 256 ? (tbl <= 2048 ? 6 : 4) : 2;
}

template <class SR, int GS, int TBL, bool NUM, int BLOCK>
__global__ void __launch_bounds__(BLOCK, hash_min_blocks(BLOCK, TBL)) k_hash(Items it, const int2* __restrict__ list, int64_t count,
                                                int64_t* __restrict__ nnz_item, const int64_t* __restrict__ Coff,
                                                int32_t* __restrict__ Cir, typename SR::T* __restrict__ Cv,
                                                int bm_words) {
    using T = typename SR::T;
    using Acc = typename SR::Acc;
    using L = HashLayout<SR, GS, TBL, NUM>;
    using G = Group<GS>;
    constexpr int NG = BLOCK / GS;
    constexpr int LOG2 = __builtin_ctz(TBL);
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = G::lane();
    const int g = G::gid();
    unsigned char* base = smem + (size_t)g * L::group;
    int32_t* keys = reinterpret_cast<int32_t*>(base);
    Acc* vals = reinterpret_cast<Acc*>(base + L::keys);
    int* s_incl = reinterpret_cast<int*>(base + L::keys + L::vals);
    int64_t* s_a0 = reinterpret_cast<int64_t*>(base + L::keys + L::vals + L::incl);
    T* s_bv = reinterpret_cast<T*>(base + L::keys + L::vals + L::incl + L::a0);
    int* s_scan = reinterpret_cast<int*>(base + L::keys + L::vals + L::incl + L::a0 + L::bv);
    int* s_cnt = s_scan + 33;
    volatile int32_t* vkeys = keys;
    // Numeric tables order their output through a row bitmap (one per group) when
    // the rows fit; otherwise they compact and sort.
    uint32_t* bitmap = reinterpret_cast<uint32_t*>(smem + (size_t)NG * L::group) + (size_t)g * bm_words;
    // per-word prefixes of the bitmap, after the bitmaps of all groups
    uint16_t* wp = reinterpret_cast<uint16_t*>(smem + (size_t)NG * L::group + (size_t)NG * bm_words * 4) +
                   (size_t)g * bm_words;
    constexpr bool CAN_BM = NUM && (GS == BLOCK || (GS == 32 && TBL >= BM_WARP_MIN_TBL));
    if constexpr (CAN_BM) {
        for (int x = lane; x < bm_words; x += GS) bitmap[x] = 0u;
    }
    // Numeric tables start empty and every column leaves its table empty again (the
    // bitmap emit resets the slots it reads; the sorting path clears the table).
    if constexpr (NUM) {
        for (int s = lane; s < TBL; s += GS) {
            keys[s] = -1;
            vals[s] = SR::zero();
        }
    }
    G::sync();

    for (int64_t w = (int64_t)blockIdx.x * NG + g; w < count; w += (int64_t)gridDim.x * NG) {
        const int2 e = __ldg(list + w);
        const Prod* pr = it.prods + e.x;
        const int64_t u = __ldg(it.item_base + e.x) + e.y;
        const int64_t bs = __ldg(pr->B.cp + e.y), be = __ldg(pr->B.cp + e.y + 1);
        if constexpr (!NUM) {
            for (int s = lane; s < TBL; s += GS) keys[s] = -1;
            if (lane == 0) *s_cnt = 0;
            G::sync();
        }
        int mycnt = 0;
        // numeric columns whose rows fit the bitmap mark a row when they claim its slot
        int mark_nw = 0;
        if constexpr (CAN_BM) {
            const int64_t mw = (pr->A.m + 31) >> 5;
            mark_nw = mw <= bm_words ? (int)mw : 0;
        }
        for (int64_t b0 = bs; b0 < be; b0 += GS) {
            const int64_t t = b0 + lane;
            int len = 0;
            int64_t a0 = 0;
            T bv = T(0);
            if (t < be) {
                int32_t k = __ldg(pr->B.ir + t);
                int64_t s, en;
                a_col(it, pr, t, k, s, en);
                a0 = s;
                len = (int)(en - s);
                if constexpr (NUM) bv = load_val<SR>(pr->B, t);
            }
            // Every member finished the previous chunk's expansion before the scan's
            // barrier (or the warp's shuffles), so the chunk arrays can be rewritten
            // after it without a closing barrier.
            int total;
            int ns = GS;   // segments in s_incl / s_a0 / s_bv
            if constexpr (GS == 32) {
                const int incl = group_incl_scan_open<GS>(len, s_scan, total);
                s_incl[lane] = incl;
                s_a0[lane] = a0;
                if constexpr (NUM) s_bv[lane] = bv;
            } else {
                // several warps: keep the nonempty segments only (their ends are then
                // distinct), so that a warp finds its products' segments by windows
                long long tot64;
                const long long inc64 = group_incl_scan64_open<GS>(len > 0 ? ((1ll << 32) | len) : 0ll,
                                                                   reinterpret_cast<long long*>(s_scan), tot64);
                if (len > 0) {
                    const int p = (int)(inc64 >> 32) - 1;
                    s_incl[p] = (int)(inc64 & 0xffffffffll);
                    s_a0[p] = a0;
                    if constexpr (NUM) s_bv[p] = bv;
                }
                ns = (int)(tot64 >> 32);
                total = (int)(tot64 & 0xffffffffll);
            }
            G::sync();
            const int32_t* __restrict__ air = pr->A.ir;
            // U products per lane per round: their loads are all issued before the first insert
            constexpr int U = 4;
            // several warps: each takes a contiguous slice of the products, in windows of 32
            int q0 = 0, qend = total, o0 = 0;
            constexpr int QSTEP = GS == 32 ? GS * U : 32 * U;
            if constexpr (GS > 32) {
                constexpr int NWG = GS / 32;
                const int wg = (threadIdx.x % GS) >> 5;
                const int C = (total + NWG * 32 - 1) / (NWG * 32) * 32;
                q0 = wg * C;
                qend = min(total, q0 + C);
                int lo = 0, hi = ns;   // segments ending at or before the slice start
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (s_incl[mid] <= q0) lo = mid + 1;
                    else hi = mid;
                }
                o0 = lo;
            }
            for (; q0 < qend; q0 += QSTEP) {
                int32_t row[U];
                T av[U];
                int seg[U];
#pragma unroll
                for (int i = 0; i < U; ++i) {
                    row[i] = -1;
                    if constexpr (GS == 32) {
                        const int q = q0 + i * GS + lane;
                        if (q < total) {
                            int lo = 0, hi = GS - 1;
                            while (lo < hi) {
                                int mid = (lo + hi) >> 1;
                                if (s_incl[mid] > q) hi = mid;
                                else lo = mid + 1;
                            }
                            const int64_t idx = s_a0[lo] + (q - (lo ? s_incl[lo - 1] : 0));
                            row[i] = __ldg(air + idx);
                            if constexpr (NUM) av[i] = load_val<SR>(pr->A, idx);
                            seg[i] = lo;
                        }
                    } else {
                        const int xw = q0 + 32 * i;
                        const int oi = warp_window_segment(s_incl, ns, xw, o0);
                        const int q = xw + (threadIdx.x & 31);   // this warp's lane, not the group's
                        if (q < qend) {
                            const int64_t idx = s_a0[oi] + (q - (oi ? s_incl[oi - 1] : 0));
                            row[i] = __ldg(air + idx);
                            if constexpr (NUM) av[i] = load_val<SR>(pr->A, idx);
                            seg[i] = oi;
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < U; ++i) {
                    if (row[i] < 0) continue;
                    const int32_t r = row[i];
                    uint32_t h = hash_row(r) >> (32 - LOG2);
                    while (true) {
                        int32_t cur = vkeys[h];
                        if (cur == r) break;
                        if (cur == -1) {
                            int32_t prev = atomicCAS(&keys[h], -1, r);
                            if (prev == -1) {
                                ++mycnt;
                                if constexpr (CAN_BM)
                                    if ((r >> 5) < mark_nw) atomicOr(&bitmap[r >> 5], 1u << (r & 31));
                                break;
                            }
                            if (prev == r) break;
                        }
                        h = (h + 1) & (TBL - 1);
                    }
                    if constexpr (NUM) SR::atomic_add(&vals[h], SR::mul(av[i], s_bv[seg[i]]));
                }
            }
            if constexpr (GS == 32) __syncwarp();
        }
        G::sync();
        if constexpr (!NUM) {
            int c = warp_sum(mycnt);
            if constexpr (GS == 32) {
                if (lane == 0) nnz_item[u] = c;
            } else {
                if ((threadIdx.x & 31) == 0) atomicAdd(s_cnt, c);
                __syncthreads();
                if (lane == 0) nnz_item[u] = *s_cnt;
            }
            G::sync();
        } else {
            // exact mode: Coff holds exact offsets.  Predicted mode (nnz_item != nullptr): Coff holds
            // capacity offsets; the exact count is recorded and the column is written only if it fits.
            const int64_t out0 = __ldg(Coff + u);
            const int64_t capn = __ldg(Coff + u + 1) - out0;
            const int32_t rb = out_row_base(pr, e.y);
            if constexpr (CAN_BM) {
                // a warp prefers the bitmap once sorting the entries would cost more than scanning it
                bool use_bm = mark_nw > 0;
                if constexpr (GS == 32) use_bm = use_bm && mark_nw <= 8 * warp_sum(mycnt);
                if (use_bm) {
                    const int total = rank_emit<SR, TBL, GS>(bitmap, wp, mark_nw, keys, vals, s_incl, s_scan,
                                                             nnz_item != nullptr, capn, out0, rb, Cir, Cv);
                    if (nnz_item && lane == 0) nnz_item[u] = total;
                    continue;
                }
                // sorting instead: drop the marks
                for (int x = lane; x < mark_nw; x += GS) bitmap[x] = 0u;
            }
            // in-place compaction toward the front: the i-th occupied slot moves to i <= its slot.
            // Each lane holds a contiguous run of S slots in registers; rounds go up the table, and
            // every destination lies below the slots of later rounds, so nothing unread is overwritten.
            constexpr int S = (TBL / GS) < 8 ? (TBL / GS) : 8;
            int pos = 0;
            for (int r0 = 0; r0 < TBL; r0 += GS * S) {
                const int base_s = r0 + lane * S;
                int32_t kk[S];
                Acc vv[S];
                int occ = 0;
#pragma unroll
                for (int i = 0; i < S; ++i) {
                    kk[i] = keys[base_s + i];
                    vv[i] = vals[base_s + i];
                    occ += kk[i] != -1;
                }
                int total;
                int o = pos + group_incl_scan<GS>(occ, s_scan, total) - occ;
                G::sync();
#pragma unroll
                for (int i = 0; i < S; ++i) {
                    if (kk[i] != -1) {
                        keys[o] = kk[i];
                        vals[o] = vv[i];
                        ++o;
                    }
                }
                pos += total;
                G::sync();
            }
            const int nnz = nnz_item ? pos : (int)capn;
            if (nnz_item) {
                if (lane == 0) nnz_item[u] = pos;
                if (pos > capn) {   // overflow: recomputed into its exact place afterwards
                    for (int s = lane; s < TBL; s += GS) {
                        keys[s] = -1;
                        vals[s] = SR::zero();
                    }
                    G::sync();
                    continue;
                }
            }
            int P = 1;
            while (P < nnz) P <<= 1;
            for (int s = nnz + lane; s < P; s += GS) keys[s] = INT_MAX;
            G::sync();
            bitonic_sort<GS>(keys, vals, P);
            for (int s = lane; s < nnz; s += GS) {
                Cir[out0 + s] = keys[s] + rb;
                Cv[out0 + s] = SR::out(vals[s]);
            }
            G::sync();
            for (int s = lane; s < TBL; s += GS) {
                keys[s] = -1;
                vals[s] = SR::zero();
            }
            G::sync();
        }
    }
}

template <class SR, int GS, int TBL, bool NUM, int BLOCK>
static void run_hash(cudaStream_t st, const Items& it, const int2* list, int64_t count, int64_t* nnz_item,
                     const int64_t* Coff, int32_t* Cir, typename SR::T* Cv) {
    if (count <= 0) return;
    using L = HashLayout<SR, GS, TBL, NUM>;
    constexpr int NG = BLOCK / GS;
    constexpr bool CAN_BM = NUM && (GS == BLOCK || (GS == 32 && TBL >= BM_WARP_MIN_TBL));
    // small groups keep the bitmap to the rows a warp would (its scan is per column)
    constexpr int64_t bm_rows = GS < 256 ? BM_WARP_MAX_ROWS : BM_MAX_ROWS;
    const int bm_words = CAN_BM && it.max_m > 0 && it.max_m <= bm_rows ? (int)((it.max_m + 31) / 32) : 0;
    size_t smem = L::group * NG + (size_t)bm_words * 6 * NG;   // bitmap words and their 16-bit prefixes
    auto kern = k_hash<SR, GS, TBL, NUM, BLOCK>;
    smem_at_least((const void*)kern, smem);
    int64_t want = ceil_div64(count, NG);
    int grid = (int)std::min<int64_t>(want, sm_count() * 32);
    kern<<<grid, BLOCK, smem, st>>>(it, list, count, nnz_item, Coff, Cir, Cv, bm_words);
    note_launch();
}

// Symbolic count of columns whose rows fit a per-group bitmap (every A_i has at
// most BM_COUNT_MAX_ROWS rows, as the SUMMA merge columns): each product sets its
// row's bit and nnz is the popcount; no keys, no probing, no table to clear.
constexpr int64_t BM_COUNT_MAX_ROWS = 32768;
// shared memory of one counting group before the bitmaps: a0, incl, scan (34), l1 (32)
template <int GS>
constexpr size_t bitcount_group_bytes() { return ((size_t)GS * 12 + 34 * 4 + 32 * 4 + 15) / 16 * 16; }
template <int GS, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 2048 / BLOCK) k_bitcount(Items it, const int2* __restrict__ list,
                                                                  int64_t count, int64_t* __restrict__ nnz_item,
                                                                  int bm_words) {
    using G = Group<GS>;
    constexpr int NG = BLOCK / GS;
    constexpr size_t GROUP = bitcount_group_bytes<GS>();
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = G::lane(), g = G::gid();
    unsigned char* base = smem + (size_t)g * GROUP;
    int64_t* s_a0 = reinterpret_cast<int64_t*>(base);
    int* s_incl = reinterpret_cast<int*>(base + (size_t)GS * 8);
    int* s_scan = s_incl + GS;
    uint32_t* l1 = reinterpret_cast<uint32_t*>(s_scan + 34);   // nonempty bitmap words (bm_words <= 1024)
    uint32_t* bitmap = reinterpret_cast<uint32_t*>(smem + (size_t)NG * GROUP) + (size_t)g * bm_words;
    for (int x = lane; x < bm_words; x += GS) bitmap[x] = 0u;
    for (int x = lane; x < 32; x += GS) l1[x] = 0u;
    G::sync();
    for (int64_t w = (int64_t)blockIdx.x * NG + g; w < count; w += (int64_t)gridDim.x * NG) {
        const int2 e = __ldg(list + w);
        const Prod* pr = it.prods + e.x;
        const int64_t u = __ldg(it.item_base + e.x) + e.y;
        const int64_t bs = __ldg(pr->B.cp + e.y), be = __ldg(pr->B.cp + e.y + 1);
        const uint32_t mrows = (uint32_t)(pr->A.m < (int64_t)bm_words * 32 ? pr->A.m : (int64_t)bm_words * 32);
        const int32_t* __restrict__ air = pr->A.ir;
        int c = 0;   // rows this lane marked first
        for (int64_t b0 = bs; b0 < be; b0 += GS) {
            const int64_t t = b0 + lane;
            int len = 0;
            int64_t a0 = 0;
            if (t < be) {
                int64_t s, en;
                a_col(it, pr, t, __ldg(pr->B.ir + t), s, en);
                a0 = s;
                len = (int)(en - s);
            }
            int total;
            int ns = GS;
            if constexpr (GS == 32) {
                const int incl = group_incl_scan_open<GS>(len, s_scan, total);
                s_incl[lane] = incl;
                s_a0[lane] = a0;
            } else {   // nonempty segments only, for the windowed walk below
                long long tot64;
                const long long inc64 = group_incl_scan64_open<GS>(len > 0 ? ((1ll << 32) | len) : 0ll,
                                                                   reinterpret_cast<long long*>(s_scan), tot64);
                if (len > 0) {
                    const int p = (int)(inc64 >> 32) - 1;
                    s_incl[p] = (int)(inc64 & 0xffffffffll);
                    s_a0[p] = a0;
                }
                ns = (int)(tot64 >> 32);
                total = (int)(tot64 & 0xffffffffll);
            }
            G::sync();
            constexpr int U = 4;
            int q0 = 0, qend = total, o0 = 0;
            constexpr int QSTEP = GS == 32 ? GS * U : 32 * U;
            if constexpr (GS > 32) {   // a contiguous slice of the products per warp
                constexpr int NWG = GS / 32;
                const int wg = (threadIdx.x % GS) >> 5;
                const int C = (total + NWG * 32 - 1) / (NWG * 32) * 32;
                q0 = wg * C;
                qend = min(total, q0 + C);
                int lo = 0, hi = ns;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (s_incl[mid] <= q0) lo = mid + 1;
                    else hi = mid;
                }
                o0 = lo;
            }
            for (; q0 < qend; q0 += QSTEP) {
                int32_t row[U];
#pragma unroll
                for (int i = 0; i < U; ++i) {
                    row[i] = -1;
                    if constexpr (GS == 32) {
                        const int q = q0 + i * GS + lane;
                        if (q < total) {
                            int lo = 0, hi = GS - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi) >> 1;
                                if (s_incl[mid] > q) hi = mid;
                                else lo = mid + 1;
                            }
                            row[i] = __ldg(air + s_a0[lo] + (q - (lo ? s_incl[lo - 1] : 0)));
                        }
                    } else {
                        const int xw = q0 + 32 * i;
                        const int oi = warp_window_segment(s_incl, ns, xw, o0);
                        const int q = xw + (threadIdx.x & 31);   // this warp's lane, not the group's
                        if (q < qend) row[i] = __ldg(air + s_a0[oi] + (q - (oi ? s_incl[oi - 1] : 0)));
                    }
                }
            // the atomic's return value says whether the row is new; a word that becomes
            // nonempty is marked in l1, so only touched words are cleared afterwards
#pragma unroll
                for (int i = 0; i < U; ++i) {
                    if ((uint32_t)row[i] >= mrows) continue;
                    const int wd = row[i] >> 5;
                    const uint32_t bit = 1u << (row[i] & 31);
                    const uint32_t old = atomicOr(&bitmap[wd], bit);
                    c += (old & bit) == 0u;
                    if (old == 0u) atomicOr(&l1[wd >> 5], 1u << (wd & 31));
                }
            }
            if constexpr (GS == 32) __syncwarp();
        }
        G::sync();
        int tot;
        group_incl_scan<GS>(c, s_scan, tot);
        if (lane == 0) nnz_item[u] = tot;
        // empty the words this column touched (through the first-level bitmap)
        for (int x = lane; x < 32; x += GS) {
            uint32_t bits = l1[x];
            while (bits) {
                bitmap[x * 32 + __ffs(bits) - 1] = 0u;
                bits &= bits - 1;
            }
            l1[x] = 0u;
        }
        G::sync();
    }
}

template <int GS, int BLOCK>
static void run_bitcount(cudaStream_t st, const Items& it, const int2* list, int64_t count, int64_t* nnz_item) {
    if (count <= 0) return;
    constexpr int NG = BLOCK / GS;
    constexpr size_t GROUP = bitcount_group_bytes<GS>();
    const int bm_words = (int)((it.max_m + 31) / 32);
    const size_t smem = (GROUP + (size_t)bm_words * 4) * NG;
    auto kern = k_bitcount<GS, BLOCK>;
    smem_at_least((const void*)kern, smem);
    const int grid = (int)std::min<int64_t>(ceil_div64(count, NG), sm_count() * 32);
    kern<<<grid, BLOCK, smem, st>>>(it, list, count, nnz_item, bm_words);
    note_launch();
}

// Tiny columns (flops <= TINY_MAX): one thread gathers the products in
// registers, insertion-sorts them by row (stable, so equal rows keep ascending
// k order), sums duplicates and writes the column.  No table, no barrier.
template <class SR, bool NUM>
__global__ void __launch_bounds__(256) k_tiny(Items it, const int2* __restrict__ list, int64_t count,
                                              int64_t* __restrict__ nnz_item, const int64_t* __restrict__ Coff,
                                              int32_t* __restrict__ Cir, typename SR::T* __restrict__ Cv) {
    using Acc = typename SR::Acc;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < count; w += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = __ldg(list + w);
        const Prod* pr = it.prods + e.x;
        const int64_t u = __ldg(it.item_base + e.x) + e.y;
        const int64_t bs = __ldg(pr->B.cp + e.y), be = __ldg(pr->B.cp + e.y + 1);
        int32_t r[TINY_MAX];
        Acc v[TINY_MAX];
        int n = 0;
        for (int64_t t = bs; t < be; ++t) {
            const int32_t k = __ldg(pr->B.ir + t);
            int64_t s0, en;
            a_col(it, pr, t, k, s0, en);
            typename SR::T bv = typename SR::T(0);
            if constexpr (NUM) bv = load_val<SR>(pr->B, t);
            for (int64_t q = s0; q < en && n < TINY_MAX; ++q) {
                r[n] = __ldg(pr->A.ir + q);
                if constexpr (NUM) v[n] = SR::mul(load_val<SR>(pr->A, q), bv);
                ++n;
            }
        }
        for (int i = 1; i < n; ++i) {
            const int32_t key = r[i];
            Acc val = NUM ? v[i] : Acc(0);
            int j = i - 1;
            while (j >= 0 && r[j] > key) {
                r[j + 1] = r[j];
                if constexpr (NUM) v[j + 1] = v[j];
                --j;
            }
            r[j + 1] = key;
            if constexpr (NUM) v[j + 1] = val;
        }
        int m = 0;
        for (int i = 0; i < n; ++i) {
            if (m > 0 && r[m - 1] == r[i]) {
                if constexpr (NUM) v[m - 1] = SR::add(v[m - 1], v[i]);
            } else {
                r[m] = r[i];
                if constexpr (NUM) v[m] = v[i];
                ++m;
            }
        }
        if constexpr (!NUM) {
            nnz_item[u] = m;
        } else {
            // exact mode: Coff are exact offsets; predicted mode (nnz_item set): capacity offsets
            const int64_t out0 = __ldg(Coff + u);
            if (nnz_item) nnz_item[u] = m;
            // overflow (predicted mode): redone in its exact place; in exact mode the counts
            // agree, and the check keeps an inconsistent input inside its column
            if (m > __ldg(Coff + u + 1) - out0) continue;
            const int32_t rb = out_row_base(pr, e.y);
            for (int i = 0; i < m; ++i) {
                Cir[out0 + i] = r[i] + rb;
                Cv[out0 + i] = SR::out(v[i]);
            }
        }
    }
}

template <class SR, bool NUM>
static void run_tiny(cudaStream_t st, const Items& it, const int2* list, int64_t count, int64_t* nnz_item,
                     const int64_t* Coff, int32_t* Cir, typename SR::T* Cv) {
    if (count <= 0) return;
    const int grid = (int)std::min<int64_t>(ceil_div64(count, 256), sm_count() * 16);
    k_tiny<SR, NUM><<<grid, 256, 0, st>>>(it, list, count, nnz_item, Coff, Cir, Cv);
    note_launch();
}

// every A_i has at most BLOCK_TIER_MAX_ROWS rows: numeric passes run in the block tier
static bool block_mode(const Items& it) { return it.max_m > 0 && it.max_m <= BLOCK_TIER_MAX_ROWS; }

template <class SR, bool NUM>
static void run_hash_bins(cudaStream_t st, const Items& it, const int2* list, const int64_t* off, const int64_t* cnt,
                          int64_t* nnz_item, const int64_t* Coff, int32_t* Cir, typename SR::T* Cv) {
    constexpr int W0 = BIN_WARP0, B0 = BIN_BLK0;
    run_tiny<SR, NUM>(st, it, list + off[BIN_TINY], cnt[BIN_TINY], nnz_item, Coff, Cir, Cv);
    run_hash<SR, 32, 64, NUM, WARP_BLOCK>(st, it, list + off[W0], cnt[W0], nnz_item, Coff, Cir, Cv);
    run_hash<SR, 32, 128, NUM, WARP_BLOCK>(st, it, list + off[W0 + 1], cnt[W0 + 1], nnz_item, Coff, Cir, Cv);
    if constexpr (!NUM) {
        if (it.max_m > 0 && it.max_m <= BM_COUNT_MAX_ROWS) {
            // rows fit a small bitmap: count the longer columns by bits (64 and 128
            // slots hold so few rows that clearing a bitmap would cost more)
            // one warp per column for the CTA-table bins too: a column of a few thousand
            // products has no barrier chain to wait on, and its bitmap is the same size
            run_bitcount<32, WARP_BLOCK>(st, it, list + off[W0 + 2],
                                         cnt[W0 + 2] + cnt[W0 + 3] + cnt[W0 + 4] + cnt[B0] + cnt[B0 + 1] + cnt[B0 + 2],
                                         nnz_item);
            return;
        }
    }
    run_hash<SR, 32, 256, NUM, WARP_BLOCK>(st, it, list + off[W0 + 2], cnt[W0 + 2], nnz_item, Coff, Cir, Cv);
    if constexpr (NUM) {
        // numeric tables of 512 and 1024 slots: one table per 2 or 4 warps, so that
        // shared memory admits more warps per SM (a warp each left a quarter of them)
        run_hash<SR, 64, 512, NUM, 64>(st, it, list + off[W0 + 3], cnt[W0 + 3], nnz_item, Coff, Cir, Cv);
        run_hash<SR, 128, 1024, NUM, 128>(st, it, list + off[W0 + 4], cnt[W0 + 4], nnz_item, Coff, Cir, Cv);
    } else {
        run_hash<SR, 32, 512, NUM, WARP_BLOCK>(st, it, list + off[W0 + 3], cnt[W0 + 3], nnz_item, Coff, Cir, Cv);
        run_hash<SR, 32, 1024, NUM, 128>(st, it, list + off[W0 + 4], cnt[W0 + 4], nnz_item, Coff, Cir, Cv);
    }
    run_hash<SR, 256, 2048, NUM, 256>(st, it, list + off[B0], cnt[B0], nnz_item, Coff, Cir, Cv);
    // 4096-slot tables: 256 threads per column when the row bitmap is small (more columns
    // in flight per SM), 512 when a large bitmap already limits the CTAs per SM
    if (it.max_m <= 65536)
        run_hash<SR, 256, 4096, NUM, 256>(st, it, list + off[B0 + 1], cnt[B0 + 1], nnz_item, Coff, Cir, Cv);
    else
        run_hash<SR, 512, 4096, NUM, 512>(st, it, list + off[B0 + 1], cnt[B0 + 1], nnz_item, Coff, Cir, Cv);
    run_hash<SR, 512, 8192, NUM, 512>(st, it, list + off[B0 + 2], cnt[B0 + 2], nnz_item, Coff, Cir, Cv);
}

// ------------------------------------------------------------------ slab tier (long columns)
// A long output column is split into P row slabs of at most RB rows (balanced by
// flops, at most MAX_PARTS, fewer where B(:,j) is long: every slab repeats two
// binary searches per entry of B(:,j)).  The symbolic kernel marks the rows of a
// slab in a shared-memory bitmap with one flattened walk over the slab's products,
// counts them and stores the slab's row set for the numeric pass: its bitmap words
// when the slab holds at least one row per word, else its rows in ascending order,
// whichever is smaller.  The numeric kernel reloads the row set into a
// shared-memory bitmap, ranks rows by per-group prefix counts (4 words = 128 rows
// per group), writes C's rows for the slab, sets the slab's values to the
// semiring zero and walks the products again, adding each one into C at its row's
// rank with an L2 reduction.  There is no shared-memory accumulator (FP64 shared
// atomics are the slow path on this part), no hashing and no sort, and a slab's
// products are spread evenly over the CTA's warps.
constexpr int RT_BLOCK = 512;

__device__ __forceinline__ int32_t lower_bound_rows(const int32_t* __restrict__ r, int64_t len, int64_t v) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)__ldg(r + mid) < v) lo = mid + 1;
        else hi = mid;
    }
    return (int32_t)lo;
}

// rows [R0, R1) of slab q of P over m rows (32-aligned cuts)
__host__ __device__ __forceinline__ void slab_rows(int64_t m, int q, int P, int64_t& R0, int64_t& R1) {
    R0 = ((int64_t)q * m / P) & ~int64_t(31);
    R1 = q == P - 1 ? m : (((int64_t)(q + 1) * m / P) & ~int64_t(31));
}

// the most rows any of the P slabs over m rows holds
__host__ __device__ __forceinline__ int64_t slab_max_rows(int64_t m, int P) {
    int64_t mx = 0;
    for (int q = 0; q < P; ++q) {
        int64_t R0, R1;
        slab_rows(m, q, P, R0, R1);
        mx = R1 - R0 > mx ? R1 - R0 : mx;
    }
    return mx;
}

// Slabs of the long columns: P per column, items[sbase[d] + q] = (d, q); the
// storage bound of the slab row sets, sum over columns of min(flops, words),
// accumulates in *store_bound (a slab stores min(words, rows) 4-byte entries and
// rows <= flops).
__global__ void k_dense_items(Items it, const int2* __restrict__ dlist, int64_t nd, const int64_t* __restrict__ flops,
                              int part_flops, int RB, int2* items, unsigned long long* nitems, int8_t* nparts,
                              int32_t* sbase, unsigned long long* store_bound, int64_t* bbase,
                              unsigned long long* bnd_total) {
    int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nd) return;
    const int2 e = dlist[d];
    const Prod* pr = it.prods + e.x;
    const int64_t f = flops[__ldg(it.item_base + e.x) + e.y];
    const int64_t deg = __ldg(pr->B.cp + e.y + 1) - __ldg(pr->B.cp + e.y);
    const int64_t m = pr->A.m;
    // slab rows stay <= RB: the fewest slabs whose 32-aligned cuts all fit (the host
    // sized RB so that MAX_PARTS slabs always do)
    int64_t pmin = m <= RB ? 1 : ceil_div64(m, (int64_t)RB);
    while (pmin < MAX_PARTS && slab_max_rows(m, (int)pmin) > RB) ++pmin;
    int64_t P = ceil_div64(f, part_flops);
    const int64_t pdeg = f / (32 * (deg > 0 ? deg : 1));   // about 32 products per (slab, B entry) at least
    P = P < pdeg ? P : pdeg;
    P = P < pmin ? pmin : P;
    P = P > MAX_PARTS ? MAX_PARTS : P;
    P = P < 1 ? 1 : P;
    nparts[d] = (int8_t)P;
    int64_t words = 0;
    for (int q = 0; q < P; ++q) {
        int64_t R0, R1;
        slab_rows(m, q, (int)P, R0, R1);
        words += (R1 - R0 + 31) >> 5;
    }
    atomicAdd(store_bound, (unsigned long long)(f < words ? f : words));
    // boundary table: P + 1 rows of deg positions (where each slab starts in every A(:,k)),
    // then two rows with where every A(:,k) starts (low and high 32 bits)
    bbase[d] = (int64_t)atomicAdd(bnd_total, (unsigned long long)((P + 3) * deg));
    unsigned long long base = atomicAdd(nitems, (unsigned long long)P);
    sbase[d] = (int32_t)base;
    for (int q = 0; q < P; ++q) items[base + q] = make_int2((int)d, q);
}

void launch_dense_items(cudaStream_t st, const Items& it, const int2* dense_list, int64_t ndense, const int64_t* flops,
                        int part_flops, int RB, int2* items, unsigned long long* nitems, int8_t* nparts,
                        int32_t* sbase, unsigned long long* store_bound, int64_t* bbase,
                        unsigned long long* bnd_total) {
    if (ndense == 0) return;
    k_dense_items<<<(int)ceil_div64(ndense, 256), 256, 0, st>>>(it, dense_list, ndense, flops, part_flops, RB, items,
                                                               nitems, nparts, sbase, store_bound, bbase, bnd_total);
    note_launch();
}

// Slab boundaries, once for both passes: row q of column d's table holds, for every
// entry t of B(:,j), where slab q starts inside A(:,k) (relative to the column's
// start); row P holds A(:,k)'s length.  One CTA per slab, every search of the slab
// in flight at once (the passes that read them no longer wait on search chains at
// their barriers).
__global__ void __launch_bounds__(256) k_slab_bounds(Items it, DenseWork dw) {
    const int64_t nsym = (int64_t)*dw.nitems;
    for (int64_t w = blockIdx.x; w < nsym; w += gridDim.x) {
        const int2 itm = dw.items[w];
        const int d = itm.x, q = itm.y;
        const int2 e = __ldg(dw.dlist + d);
        const Prod* pr = it.prods + e.x;
        const int P = dw.nparts[d];
        const int64_t m = pr->A.m;
        int64_t R0, R1;
        slab_rows(m, q, P, R0, R1);
        const int64_t bs = __ldg(pr->B.cp + e.y), be = __ldg(pr->B.cp + e.y + 1);
        const int64_t deg = be - bs;
        int32_t* __restrict__ row = dw.bnd + dw.bbase[d] + (int64_t)q * deg;
        const int32_t* __restrict__ air = pr->A.ir;
        if (threadIdx.x == 0) {
            SlabRec r;
            r.prod = e.x;
            r.col = e.y;
            r.r0 = (int32_t)R0;
            r.r1 = (int32_t)R1;
            r.rb = out_row_base(pr, e.y);
            r.cnt = 0;
            r.bs = bs;
            r.be = be;
            r.bnd = dw.bbase[d] + (int64_t)q * deg;
            r.u = __ldg(it.item_base + e.x) + e.y;
            r.ob = 0;
            r.soff = -1;
            r.sab = dw.bbase[d] + (int64_t)(P + 1) * deg;
            dw.rec[w] = r;
        }
        for (int64_t t = threadIdx.x; t < deg; t += blockDim.x) {
            const int32_t k = __ldg(pr->B.ir + bs + t);
            int64_t s, en;
            a_col(it, pr, bs + t, k, s, en);
            row[t] = q == 0 ? 0 : lower_bound_rows(air + s, en - s, R0);
            if (q == P - 1) row[t + deg] = (int32_t)(en - s);
            if (q == 0) {   // where A(:,k) starts, for the passes' segment arithmetic
                int32_t* sr = dw.bnd + dw.bbase[d] + (int64_t)(P + 1) * deg;
                sr[t] = (int32_t)(uint32_t)s;
                sr[t + deg] = (int32_t)(s >> 32);
            }
        }
    }
}

// flag = 1 when some stored value of an operand is false (boolean semiring): then
// the numeric pass must evaluate the products; else every output value is true.
__global__ void k_false_values(Items it, int* flag) {
    for (int64_t p = blockIdx.y; p < it.nprod; p += gridDim.y) {
        const Prod* pr = it.prods + p;
        for (int side = 0; side < 2; ++side) {
            const DMat& M = side ? pr->B : pr->A;
            if (M.num == nullptr || M.nzc <= 0) continue;
            const uint8_t* __restrict__ v = reinterpret_cast<const uint8_t*>(M.num);
            const int64_t stride = (int64_t)gridDim.x * blockDim.x;
            const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
            bool f = false;
            if (M.ce) {   // a CSC with gaps: only the stored part of every column
                for (int64_t c = t0; c < M.nzc; c += stride)
                    for (int64_t i = __ldg(M.cp + c); i < __ldg(M.ce + c); ++i) f |= __ldg(v + i) == 0;
            } else {
                const int64_t s = __ldg(M.cp), e = __ldg(M.cp + M.nzc);
                for (int64_t i = s + t0; i < e; i += stride) f |= __ldg(v + i) == 0;
            }
            if (f) *flag = 1;
        }
    }
}

__global__ void k_any_false(const uint8_t* __restrict__ v, int64_t n, int* flag) {
    bool f = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        f |= __ldg(v + i) == 0;
    if (f) *flag = 1;
}

void launch_any_false(cudaStream_t st, const void* vals, int64_t n, int* flag) {
    if (!vals || n <= 0) return;
    k_any_false<<<(int)std::min<int64_t>(ceil_div64(n, 256), sm_count() * 8), 256, 0, st>>>((const uint8_t*)vals, n,
                                                                                          flag);
    note_launch();
}

void launch_false_values(cudaStream_t st, const Items& it, int* flag) {
    if (it.nprod <= 0) return;
    const int gy = (int)std::min<int64_t>(it.nprod, 65535);
    const int gx = std::max(1, std::min(256, 4096 / gy));
    k_false_values<<<dim3(gx, gy), 256, 0, st>>>(it, flag);
    note_launch();
}

// Inclusive scan of a 64-bit value over the CTA (RT_BLOCK threads).
__device__ __forceinline__ unsigned long long rt_block_incl_scan64(unsigned long long v, unsigned long long* ws,
                                                                   unsigned long long& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = lane < RT_BLOCK / 32 ? ws[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < RT_BLOCK / 32) ws[lane] = s;
    }
    __syncthreads();
    const unsigned long long add = w > 0 ? ws[w - 1] : 0ull;
    total = ws[RT_BLOCK / 32 - 1];
    __syncthreads();
    return x + add;
}

struct RangeSmem {   // per-batch segments of the flattened expansion (compacted: all nonempty)
    int end[RT_BLOCK];        // inclusive prefix of segment lengths (exclusive end in flattened space)
    int64_t start[RT_BLOCK];  // first position of the segment in A.ir
    int64_t bv[RT_BLOCK];     // B value bits (read back as SR::T)
    int64_t stop[RT_BLOCK];   // one past the segment's last position (quad walks)
    unsigned long long ws[32];
    int wc[RT_BLOCK / 32 + 1];
};
// shared-memory offset of what follows a RangeSmem (16-byte aligned for vector access)
constexpr size_t RS_BYTES = (sizeof(RangeSmem) + 15) / 16 * 16;

// Compacts the active (k, segment) pairs of this batch into sc and returns
// (number of segments, number of products).  Called by all threads.
__device__ __forceinline__ void rt_compact(RangeSmem* sc, bool active, int len, int64_t a, int64_t bvbits, int& ns,
                                           int& T, int64_t stop = 0) {
    const unsigned long long packed = active && len > 0 ? ((1ull << 32) | (unsigned)len) : 0ull;
    unsigned long long tot;
    const unsigned long long inc = rt_block_incl_scan64(packed, sc->ws, tot);
    if (packed) {
        const int pos = (int)(inc >> 32) - 1;
        sc->end[pos] = (int)(inc & 0xffffffffull);
        sc->start[pos] = a;
        sc->bv[pos] = bvbits;
        sc->stop[pos] = stop;
    }
    ns = (int)(tot >> 32);
    T = (int)(tot & 0xffffffffull);
    __syncthreads();
}

// Where A(:,k) starts for entry i of B(:,j) (deg entries): two int32 rows of the
// column's boundary table, low and high 32 bits, written by the boundary pre-pass.
__device__ __forceinline__ int64_t seg_start(const int32_t* __restrict__ sab, int64_t i, int64_t deg) {
    return (int64_t)(uint32_t)__ldg(sab + i) | ((int64_t)__ldg(sab + deg + i) << 32);
}

// Flattened walk over the products of rows [R0, R1) of column bs..be of B: B's
// entries in chunks of RT_BLOCK; per entry the part of A(:,k) inside the rows
// (two binary searches), compacted into segments; each warp takes a contiguous
// slice of the chunk's products, four 32-product windows per step with every load
// issued before the updates.  f(valid, row, a, b) is called by all 32 lanes of a
// warp for each window of products (a and b, the A and B values, only when NUM;
// row is INT_MIN on lanes without a product).  Ends with a CTA barrier.
template <class SR, bool NUM, class F>
__device__ __forceinline__ void slab_walk(const Items& it, const Prod* pr, int64_t bs, int64_t be,
                                          const int32_t* __restrict__ brow0, const int32_t* __restrict__ brow1,
                                          const int32_t* __restrict__ sab, RangeSmem* sc, F&& f) {
    using T = typename SR::T;
    constexpr int U = 4, NWARP = RT_BLOCK / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t* __restrict__ air = pr->A.ir;
    for (int64_t b0 = bs; b0 < be; b0 += RT_BLOCK) {
        const int64_t t = b0 + tid;
        int len = 0;
        int64_t a = 0, bvbits = 0;
        if (t < be) {
            const int64_t s = seg_start(sab, t - bs, be - bs);
            a = s + __ldg(brow0 + (t - bs));
            const int64_t b = s + __ldg(brow1 + (t - bs));
            len = (int)(b - a);
            if constexpr (NUM) *reinterpret_cast<T*>(&bvbits) = load_val<SR>(pr->B, t);
        }
        int ns, Tn;
        rt_compact(sc, t < be, len, a, bvbits, ns, Tn);
        const int C = (Tn + NWARP * 32 - 1) / (NWARP * 32) * 32;
        const int xb = warp * C, xe = min(Tn, xb + C);
        if (xb < xe) {
            int lo = 0, hi = ns;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sc->end[mid] <= xb) lo = mid + 1;
                else hi = mid;
            }
            int o0 = lo;
            for (int x0 = xb; x0 < xe; x0 += 32 * U) {
                int64_t idx[U];
                bool ok[U];
                int ob[U];
#pragma unroll
                for (int uu = 0; uu < U; ++uu) {
                    const int xw = x0 + 32 * uu;
                    const int oi = warp_window_segment(sc->end, ns, xw, o0);
                    ok[uu] = xw + lane < xe;
                    ob[uu] = oi;
                    idx[uu] = ok[uu] ? sc->start[oi] + (xw + lane - (oi ? sc->end[oi - 1] : 0)) : 0;
                }
                int32_t row[U];
                T av[U];
#pragma unroll
                for (int uu = 0; uu < U; ++uu) {
                    row[uu] = ok[uu] ? __ldg(air + idx[uu]) : INT_MIN;
                    if constexpr (NUM) av[uu] = ok[uu] ? load_val<SR>(pr->A, idx[uu]) : T(0);
                }
#pragma unroll
                for (int uu = 0; uu < U; ++uu) {
                    if constexpr (NUM) f(ok[uu], row[uu], av[uu], ok[uu] ? *reinterpret_cast<const T*>(&sc->bv[ob[uu]]) : T(0));
                    else f(ok[uu], row[uu], T(0), T(0));
                }
            }
        }
        __syncthreads();
    }
}

// Four consecutive values of A at an aligned position p (16-byte loads: one for
// 4- and 1-byte types, two for 8-byte types).
template <class T>
__device__ __forceinline__ void load4(const T* __restrict__ p, T v[4]) {
    if constexpr (sizeof(T) == 8) {
        const ulonglong2 x = __ldg(reinterpret_cast<const ulonglong2*>(p));
        const ulonglong2 y = __ldg(reinterpret_cast<const ulonglong2*>(p) + 1);
        const unsigned long long w[4] = {x.x, x.y, y.x, y.y};
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = *reinterpret_cast<const T*>(&w[j]);
    } else if constexpr (sizeof(T) == 4) {
        const uint4 x = __ldg(reinterpret_cast<const uint4*>(p));
        const unsigned w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = *reinterpret_cast<const T*>(&w[j]);
    } else {
        const unsigned x = __ldg(reinterpret_cast<const unsigned*>(p));
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = (T)((x >> (8 * j)) & 0xffu);
    }
}

// slab_walk over aligned quads: a segment [a, b) of A(:,k) covers the quads
// q = a/4 .. (b-1)/4, and each lane takes one quad per window, loading its four
// rows with one 16-byte load (and its values with one or two) and masking the
// positions outside [a, b).  U windows per step, every load issued before the
// updates.  Needs A.ir and A.num 16-byte aligned and A a CSC whose arrays hold
// nnz_end entries (a quad past the end is read one by one).
// f(valid, row, a, b) as in slab_walk, four times per window.
template <class SR, bool NUM, int U, class F>
__device__ __forceinline__ void slab_walk_quads(const Items& it, const Prod* pr, int64_t bs, int64_t be,
                                                const int32_t* __restrict__ brow0,
                                                const int32_t* __restrict__ brow1, const int32_t* __restrict__ sab,
                                                int64_t nnz_end, RangeSmem* sc, F&& f) {
    using T = typename SR::T;
    constexpr int NWARP = RT_BLOCK / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t* __restrict__ air = pr->A.ir;
    const T* __restrict__ anum = reinterpret_cast<const T*>(pr->A.num);
    for (int64_t b0 = bs; b0 < be; b0 += RT_BLOCK) {
        const int64_t t = b0 + tid;
        int nq = 0;
        int64_t a = 0, b = 0, bvbits = 0;
        if (t < be) {
            const int64_t s = seg_start(sab, t - bs, be - bs);
            a = s + __ldg(brow0 + (t - bs));
            b = s + __ldg(brow1 + (t - bs));
            nq = b > a ? (int)(((b - 1) >> 2) - (a >> 2) + 1) : 0;
            if constexpr (NUM) *reinterpret_cast<T*>(&bvbits) = load_val<SR>(pr->B, t);
        }
        int ns, Tq;
        rt_compact(sc, t < be, nq, a, bvbits, ns, Tq, b);
        const int C = (Tq + NWARP * 32 - 1) / (NWARP * 32) * 32;
        const int xb = warp * C, xe = min(Tq, xb + C);
        if (xb < xe) {
            int lo = 0, hi = xb > 0 ? ns : 0;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sc->end[mid] <= xb) lo = mid + 1;
                else hi = mid;
            }
            int o0 = lo;
            for (int x0 = xb; x0 < xe; x0 += 32 * U) {
                int4 rq[U];
                T av[U][4];
                T bv[U];
                unsigned vm[U];   // bit j: position p0 + j lies in the segment
#pragma unroll
                for (int uu = 0; uu < U; ++uu) {
                    const int xw = x0 + 32 * uu;
                    const int oi = warp_window_segment(sc->end, ns, xw, o0);
                    rq[uu] = make_int4(INT_MIN, INT_MIN, INT_MIN, INT_MIN);
#pragma unroll
                    for (int j = 0; j < 4; ++j) av[uu][j] = T(0);
                    bv[uu] = T(0);
                    vm[uu] = 0u;
                    if (xw + lane < xe) {
                        const int64_t sa = sc->start[oi], sb = sc->stop[oi];
                        const int64_t p0 = ((sa >> 2) + (xw + lane - (oi ? sc->end[oi - 1] : 0))) << 2;
                        // sa - p0 is in [-inf, 3] and sb - p0 in [1, inf): the quad holds
                        // positions lo .. hi-1 of the segment
                        const int qlo = (int)max(sa - p0, (int64_t)0);
                        const int qhi = (int)min(sb - p0, (int64_t)4);
                        vm[uu] = (0xfu << qlo) & (0xfu >> (4 - qhi));
                        if (p0 + 4 <= nnz_end) {
                            rq[uu] = __ldg(reinterpret_cast<const int4*>(air + p0));
                            if constexpr (NUM) {
                                if (anum) load4<T>(anum + p0, av[uu]);
                                else av[uu][0] = av[uu][1] = av[uu][2] = av[uu][3] = (T)SR::one();
                            }
                        } else {   // the array's last, partial quad
                            int32_t r4[4] = {INT_MIN, INT_MIN, INT_MIN, INT_MIN};
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if (p0 + j < nnz_end) {
                                    r4[j] = __ldg(air + p0 + j);
                                    if constexpr (NUM) av[uu][j] = load_val<SR>(pr->A, p0 + j);
                                }
                            rq[uu] = make_int4(r4[0], r4[1], r4[2], r4[3]);
                        }
                        if constexpr (NUM) bv[uu] = *reinterpret_cast<const T*>(&sc->bv[oi]);
                    }
                }
#pragma unroll
                for (int uu = 0; uu < U; ++uu) {
                    const int32_t r4[4] = {rq[uu].x, rq[uu].y, rq[uu].z, rq[uu].w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool v = (vm[uu] >> j) & 1u;
                        f(v, v ? r4[j] : INT_MIN, av[uu][j], bv[uu]);
                    }
                }
            }
        }
        __syncthreads();
    }
}

// the quad walk applies to a product whose A is a CSC (no DCSC index, no gaps) with
// 16-byte aligned row and value arrays
__device__ __forceinline__ bool quads_ok(const Prod* pr) {
    return pr->A.jc == nullptr && pr->A.ce == nullptr && ((uintptr_t)pr->A.ir & 15) == 0 &&
           ((uintptr_t)pr->A.num & 15) == 0;
}

// Symbolic slab kernel: mark, count, store the row set.
__global__ void __launch_bounds__(RT_BLOCK, 2) k_slab_sym(Items it, DenseWork dw) {
    extern __shared__ __align__(16) unsigned char smem[];
    RangeSmem* sc = reinterpret_cast<RangeSmem*>(smem);
    uint32_t* bitmap = reinterpret_cast<uint32_t*>(smem + RS_BYTES);
    int* s_scan = sc->wc;
    __shared__ long long s_off;
    __shared__ SlabRec s_rec[2];   // this slab's record and the next one's, in flight
    constexpr int RC = sizeof(SlabRec) / 16;
    const int tid = threadIdx.x;
    const int64_t nsym = (int64_t)*dw.nitems;
    if (tid < RC && (int64_t)blockIdx.x < nsym)
        cp_async16(reinterpret_cast<int4*>(&s_rec[0]) + tid, reinterpret_cast<const int4*>(dw.rec + blockIdx.x) + tid);
    int k = 0;
    for (int64_t w = blockIdx.x; w < nsym; w += gridDim.x, k ^= 1) {
        if (tid < RC) cp_async_wait_all();
        __syncthreads();   // s_rec[k] is slab w's record; s_rec[k ^ 1] is free
        if (tid < RC && w + gridDim.x < nsym)
            cp_async16(reinterpret_cast<int4*>(&s_rec[k ^ 1]) + tid,
                       reinterpret_cast<const int4*>(dw.rec + w + gridDim.x) + tid);
        const SlabRec& rc = s_rec[k];
        const Prod* pr = it.prods + rc.prod;
        const int64_t R0 = rc.r0, R1 = rc.r1;
        const int nw = (int)((R1 - R0 + 31) >> 5);
        const int ng = (nw + 3) >> 2;   // groups of 4 words (the bitmap is padded to whole groups)
        const int64_t bs = rc.bs, be = rc.be;
        for (int g = tid; g < ng; g += RT_BLOCK) reinterpret_cast<uint4*>(bitmap)[g] = make_uint4(0u, 0u, 0u, 0u);
        __syncthreads();
        const int span = (int)(R1 - R0);
        const int32_t r0 = (int32_t)R0;
        // one shared atomic per product: R-MAT rows of one window mostly fall in different
        // words, so folding lanes per word first (shuffles) measured slower
        auto mark = [&](bool ok, int32_t row, uint8_t, uint8_t) {
            const int lr = row - r0;
            if (ok && (unsigned)lr < (unsigned)span) atomicOr(&bitmap[lr >> 5], 1u << (lr & 31));
        };
        const int32_t* brow0 = dw.bnd + rc.bnd;
        const int32_t* brow1 = brow0 + (be - bs);
        const int32_t* sab = dw.bnd + rc.sab;
        if (quads_ok(pr)) slab_walk_quads<BOOL8, false, 2>(it, pr, bs, be, brow0, brow1, sab, pr->A.nnz, sc, mark);
        else slab_walk<BOOL8, false>(it, pr, bs, be, brow0, brow1, sab, sc, mark);
        // count per chunk of 32 groups (lane l reads group 32 c + l with one 16-byte load:
        // no bank conflicts); a thread owns cpt consecutive chunks for the CTA scan
        constexpr int NWARP = RT_BLOCK / 32;
        const int lane = tid & 31, warp = tid >> 5;
        const int nch = (ng + 31) >> 5;
        const uint4* __restrict__ grp4 = reinterpret_cast<const uint4*>(bitmap);
        int* s_cc = reinterpret_cast<int*>(sc->start);   // the walk's segment arrays are free now
        for (int cc = warp; cc < nch; cc += NWARP) {
            const int g = cc * 32 + lane;
            int c = 0;
            if (g < ng) {
                const uint4 v = grp4[g];
                c = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
            }
            c = __reduce_add_sync(0xffffffffu, c);
            if (lane == 0) s_cc[cc] = c;
        }
        __syncthreads();
        const int cpt = (nch + RT_BLOCK - 1) / RT_BLOCK;
        const int c0 = min(tid * cpt, nch), c1 = min(c0 + cpt, nch);
        int cnt = 0;
        for (int cc = c0; cc < c1; ++cc) cnt += s_cc[cc];
        int total;
        int excl = group_incl_scan<RT_BLOCK>(cnt, s_scan, total) - cnt;
        for (int cc = c0; cc < c1; ++cc) {
            const int c = s_cc[cc];
            s_cc[cc] = excl;   // rows before chunk cc
            excl += c;
        }
        const bool dense = total >= nw;
        const int64_t size = dense ? nw : total;
        if (tid == 0) {
            long long off = size > 0 ? (long long)atomicAdd(dw.store_ctr, (unsigned long long)size) : 0;
            if (off + size > dw.store_cap) {
                atomicExch(dw.err, 3);
                off = -1;
            }
            dw.soff[w] = off;
            dw.scount[w] = total;
            dw.rec[w].soff = off;
            dw.rec[w].cnt = total;
            s_off = off;
        }
        __syncthreads();
        const long long off = s_off;
        if (off >= 0 && size > 0) {
            uint32_t* __restrict__ out = dw.store + off;
            if (dense) {
                for (int x = tid; x < nw; x += RT_BLOCK) __stcs(out + x, bitmap[x]);
            } else {
                // a warp per chunk: lanes write their group's rows at warp-scanned offsets,
                // so the lanes of one store hit neighbouring addresses
                for (int cc = warp; cc < nch; cc += NWARP) {
                    const int g = cc * 32 + lane;
                    uint4 v = make_uint4(0u, 0u, 0u, 0u);
                    if (g < ng) v = grp4[g];
                    const int c = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
                    int r = s_cc[cc] + warp_incl_scan(c) - c;
                    if (__ballot_sync(0xffffffffu, c != 0) == 0u) continue;
                    const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
                    const uint32_t base = (uint32_t)(R0 + (int64_t)g * 128);
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        uint32_t bits = wv[y];
                        while (bits) {
                            __stcs(out + r++, base + 32 * y + __ffs(bits) - 1);
                            bits &= bits - 1;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Numeric slab kernel: row set -> ranks -> C's rows, zero values, L2 reductions.
template <class SR>
__global__ void __launch_bounds__(RT_BLOCK, 2) k_slab_num(Items it, DenseWork dw, const int64_t* __restrict__ Coff,
                                                          int32_t* __restrict__ Cir, typename SR::T* __restrict__ Cv) {
    using T = typename SR::T;
    extern __shared__ __align__(16) unsigned char smem[];
    RangeSmem* sc = reinterpret_cast<RangeSmem*>(smem);
    uint32_t* bitmap = reinterpret_cast<uint32_t*>(smem + RS_BYTES);              // groups * 4 words
    int* gp = reinterpret_cast<int*>(bitmap + (size_t)(dw.RB / 128 + 1) * 4);    // rows before each group
    int* s_scan = sc->wc;
    const int tid = threadIdx.x;
    // boolean products whose operands hold no false value: every output is true
    const bool walk = SR::id != SPGEMM_OR_AND_BOOL || dw.vals_zero == nullptr || *dw.vals_zero != 0;
    const T init = walk ? SR::out(SR::zero()) : T(1);
    const int64_t nsym = (int64_t)*dw.nitems;
    __shared__ SlabRec s_rec[2];   // this slab's record and the next one's, in flight
    constexpr int RC = sizeof(SlabRec) / 16;
    if (tid < RC && (int64_t)blockIdx.x < nsym)
        cp_async16(reinterpret_cast<int4*>(&s_rec[0]) + tid, reinterpret_cast<const int4*>(dw.rec + blockIdx.x) + tid);
    int kb = 0;
    for (int64_t w = blockIdx.x; w < nsym; w += gridDim.x, kb ^= 1) {
        if (tid < RC) cp_async_wait_all();
        __syncthreads();   // s_rec[kb] is slab w's record; s_rec[kb ^ 1] is free
        if (tid < RC && w + gridDim.x < nsym)
            cp_async16(reinterpret_cast<int4*>(&s_rec[kb ^ 1]) + tid,
                       reinterpret_cast<const int4*>(dw.rec + w + gridDim.x) + tid);
        const SlabRec& rc = s_rec[kb];
        const int cnt = rc.cnt;
        // the same for every thread of the CTA; a row set that found no room (possible
        // only with malformed input, reported by the symbolic pass) is skipped
        if (cnt == 0 || rc.soff < 0) continue;
        const Prod* pr = it.prods + rc.prod;
        const int64_t R0 = rc.r0, R1 = rc.r1;
        const int nw = (int)((R1 - R0 + 31) >> 5);
        const int ng = (nw + 3) >> 2;
        const int32_t rb = rc.rb;
        const int64_t ob = rc.ob;
        const uint32_t* __restrict__ rs = dw.store + rc.soff;
        const bool dense = cnt >= nw;
        // Streaming data (the stored row sets, read once; C's rows, written once) use
        // evict-first loads and stores, so that the slab's value region, zeroed below and
        // then reduced into, stays in L2 instead of coming back from DRAM.
        // 1. the slab's row bitmap (padded to whole groups)
        if (dense) {
            for (int x = tid; x < ng * 4; x += RT_BLOCK) bitmap[x] = x < nw ? __ldcs(rs + x) : 0u;
        } else {
            for (int x = tid; x < ng * 4; x += RT_BLOCK) bitmap[x] = 0u;
            __syncthreads();
            for (int i0 = 0; i0 < cnt; i0 += RT_BLOCK) {
                const int i = i0 + tid;
                const int32_t r = i < cnt ? (int32_t)__ldcs(rs + i) : -1;
                const int lr = (int)(r - R0);
                if (i < cnt) {
                    __stcs(Cir + ob + i, r + rb);    // C's rows: the row list itself
                    atomicOr(&bitmap[lr >> 5], 1u << (lr & 31));
                }
            }
        }
        __syncthreads();
        // 2. rows before every group: a warp per chunk of 32 groups (lane l reads group
        //    32 c + l: no bank conflicts), chunk totals scanned by the CTA, then added
        constexpr int NWARP = RT_BLOCK / 32;
        const int lane = tid & 31, warp = tid >> 5;
        const int nch = (ng + 31) >> 5;
        int* s_cc = reinterpret_cast<int*>(sc->start);   // free until the walk
        for (int cc = warp; cc < nch; cc += NWARP) {
            const int g = cc * 32 + lane;
            int c = 0;
            if (g < ng) {
                const uint4 grp = reinterpret_cast<const uint4*>(bitmap)[g];
                c = __popc(grp.x) + __popc(grp.y) + __popc(grp.z) + __popc(grp.w);
            }
            const int inc = warp_incl_scan(c);
            if (g < ng) gp[g] = inc - c;
            if (lane == 31) s_cc[cc] = inc;
        }
        __syncthreads();
        {
            const int cpt = (nch + RT_BLOCK - 1) / RT_BLOCK;
            const int c0 = min(tid * cpt, nch), c1 = min(c0 + cpt, nch);
            int c = 0;
            for (int cc = c0; cc < c1; ++cc) c += s_cc[cc];
            int total;
            int excl = group_incl_scan<RT_BLOCK>(c, s_scan, total) - c;
            for (int cc = c0; cc < c1; ++cc) {
                const int v = s_cc[cc];
                s_cc[cc] = excl;
                excl += v;
            }
        }
        __syncthreads();
        for (int g = tid; g < ng; g += RT_BLOCK) gp[g] += s_cc[g >> 5];
        __syncthreads();
        // 3. C's rows of a bitmap slab: a warp per chunk of 32 groups; lanes write their
        //    group's rows from its rank base, or, for chunks of at least 16 rows a word,
        //    the warp writes one word at a time (lane l: bit l), so that every store
        //    covers neighbouring addresses
        if (dense) {
            const uint4* __restrict__ grp4 = reinterpret_cast<const uint4*>(bitmap);
            for (int cc = warp; cc < nch; cc += NWARP) {
                const int g = cc * 32 + lane;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (g < ng) v = grp4[g];
                const int c = __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
                const int tot = __reduce_add_sync(0xffffffffu, c);
                if (tot == 0) continue;
                int r = g < ng ? gp[g] : 0;
                const int32_t base = (int32_t)(R0 + (int64_t)g * 128) + rb;
                const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
                if (tot >= 2048) {
                    for (int src = 0; src < 32; ++src) {
                        int ry = __shfl_sync(0xffffffffu, r, src);
                        const int32_t by = __shfl_sync(0xffffffffu, base, src);
#pragma unroll
                        for (int y = 0; y < 4; ++y) {
                            const uint32_t wy = __shfl_sync(0xffffffffu, wv[y], src);
                            if ((wy >> lane) & 1u)
                                __stcs(Cir + ob + ry + __popc(wy & ((1u << lane) - 1u)), by + 32 * y + lane);
                            ry += __popc(wy);
                        }
                    }
                } else {
#pragma unroll
                    for (int y = 0; y < 4; ++y) {
                        uint32_t bits = wv[y];
                        while (bits) {
                            __stcs(Cir + ob + r++, base + 32 * y + __ffs(bits) - 1);
                            bits &= bits - 1;
                        }
                    }
                }
            }
        }
        // 4. values: the semiring zero (all true for the boolean shortcut)
        for (int i = tid; i < cnt; i += RT_BLOCK) Cv[ob + i] = init;
        __syncthreads();   // the stores above come before this CTA's reductions
        // 5. every product, added at its row's rank
        if (walk) {
            const int span = (int)(R1 - R0);
            const int32_t r0 = (int32_t)R0;
            auto add = [&](bool ok, int32_t row, T a, T b) {
                if (!ok) return;
                const int lr = row - r0;
                if ((unsigned)lr >= (unsigned)span) return;   // malformed input only
                const int wd = lr >> 5, g = wd >> 2, y = wd & 3;
                const uint4 grp = reinterpret_cast<const uint4*>(bitmap)[g];
                const uint32_t wv = y == 0 ? grp.x : y == 1 ? grp.y : y == 2 ? grp.z : grp.w;
                const uint32_t bit = 1u << (lr & 31);
                if (!(wv & bit)) return;                      // malformed input only
                const int rank = gp[g] + __popc(wv & (bit - 1u)) + (y > 0 ? __popc(grp.x) : 0) +
                                 (y > 1 ? __popc(grp.y) : 0) + (y > 2 ? __popc(grp.z) : 0);
                red_out<SR>(Cv, ob + rank, SR::mul(a, b));
            };
            const int64_t bs = rc.bs, be = rc.be;
            const int32_t* brow0 = dw.bnd + rc.bnd;
            const int32_t* brow1 = brow0 + (be - bs);
            const int32_t* sab = dw.bnd + rc.sab;
            if (quads_ok(pr)) slab_walk_quads<SR, true, 2>(it, pr, bs, be, brow0, brow1, sab, pr->A.nnz, sc, add);
            else slab_walk<SR, true>(it, pr, bs, be, brow0, brow1, sab, sc, add);
        } else {
            __syncthreads();
        }
    }
}

// Completes the slab records for the numeric pass: where each slab's rows start in C.
__global__ void k_slab_fin(DenseWork dw, const int64_t* __restrict__ Coff) {
    const int64_t nsym = (int64_t)*dw.nitems;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nsym; w += (int64_t)gridDim.x * blockDim.x)
        dw.rec[w].ob = __ldg(Coff + dw.rec[w].u) + dw.spref[w];
}

// CTAs per SM the kernel can keep resident with `smem` bytes, times the SM count
static int resident_grid(const void* fn, int block, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * sm_count();
}

template <class SR>
static void run_slabs(cudaStream_t st, const Items& it, const DenseWork& dw, bool numeric, const int64_t* Coff,
                      int32_t* Cir, typename SR::T* Cv) {
    if (dw.ndense <= 0) return;
    const int64_t nslab_max = dw.nslabs > 0 ? dw.nslabs : dw.ndense * MAX_PARTS;
    if (!numeric) {
        k_slab_bounds<<<(int)std::min<int64_t>(nslab_max, sm_count() * 8), 256, 0, st>>>(it, dw);
        note_launch();
        const size_t smem = RS_BYTES + (size_t)(dw.RB / 128 + 1) * 16;
        smem_at_least((const void*)k_slab_sym, smem);
        const int grid = (int)std::min<int64_t>(nslab_max, resident_grid((const void*)k_slab_sym, RT_BLOCK, smem));
        k_slab_sym<<<grid, RT_BLOCK, smem, st>>>(it, dw);
    } else {
        k_slab_fin<<<(int)std::min<int64_t>(ceil_div64(nslab_max, 256), sm_count() * 8), 256, 0, st>>>(dw, Coff);
        note_launch();
        const size_t smem = RS_BYTES + (size_t)(dw.RB / 128 + 1) * 16 + (size_t)(dw.RB / 128 + 1) * 4;
        smem_at_least((const void*)k_slab_num<SR>, smem);
        const int grid = (int)std::min<int64_t>(nslab_max, resident_grid((const void*)k_slab_num<SR>, RT_BLOCK, smem));
        k_slab_num<SR><<<grid, RT_BLOCK, smem, st>>>(it, dw, Coff, Cir, Cv);
    }
    note_launch();
}

template <class SR>
void launch_numeric_predicted(cudaStream_t st, const Items& it, const int2* list, const int64_t* bin_off,
                              const int64_t* bin_cnt, const DenseWork& dw, const int64_t* cap_off, int64_t* nnz_item,
                              int32_t* Cir, typename SR::T* Cv) {
    if (block_mode(it)) {
        run_tiny<SR, true>(st, it, list + bin_off[BIN_TINY], bin_cnt[BIN_TINY], nnz_item, cap_off, Cir, Cv);
        launch_block_tier<SR>(st, it, list, bin_off, bin_cnt, dw, nnz_item, cap_off, Cir, Cv, 1);
        return;
    }
    run_hash_bins<SR, true>(st, it, list, bin_off, bin_cnt, nnz_item, cap_off, Cir, Cv);
}

template <class SR>
void launch_symbolic(cudaStream_t st, const Items& it, TierCfg cfg, const int2* list, const int64_t* bin_off,
                     const int64_t* bin_cnt, const DenseWork& dw, int64_t* nnz_item, int which) {
    (void)cfg;
    if (which & 1) run_hash_bins<SR, false>(st, it, list, bin_off, bin_cnt, nnz_item, nullptr, nullptr, nullptr);
    if (which & 2) {
        if (dw.dcol) run_bitcount<256, 256>(st, it, dw.dlist, dw.ndense, nnz_item);   // rows fit the bitmap
        else run_slabs<SR>(st, it, dw, false, nullptr, nullptr, nullptr);
    }
}

template <class SR>
void launch_numeric(cudaStream_t st, const Items& it, TierCfg cfg, const int2* list, const int64_t* bin_off,
                    const int64_t* bin_cnt, const DenseWork& dw, const int64_t* Coff, int32_t* Cir,
                    typename SR::T* Cv, int which) {
    (void)cfg;
    if (block_mode(it)) {
        if (which & 1) run_tiny<SR, true>(st, it, list + bin_off[BIN_TINY], bin_cnt[BIN_TINY], nullptr, Coff, Cir, Cv);
        launch_block_tier<SR>(st, it, list, bin_off, bin_cnt, dw, nullptr, Coff, Cir, Cv, which);
        return;
    }
    if (which & 1) run_hash_bins<SR, true>(st, it, list, bin_off, bin_cnt, nullptr, Coff, Cir, Cv);
    if (which & 2) run_slabs<SR>(st, it, dw, true, Coff, Cir, Cv);
}

#define SG_INST(SR)                                                                                              \
    template void launch_symbolic<SR>(cudaStream_t, const Items&, TierCfg, const int2*, const int64_t*,          \
                                      const int64_t*, const DenseWork&, int64_t*, int);                          \
    template void launch_numeric<SR>(cudaStream_t, const Items&, TierCfg, const int2*, const int64_t*,           \
                                     const int64_t*, const DenseWork&, const int64_t*, int32_t*, typename SR::T*, \
                                     int);                                                                       \
    template void launch_numeric_predicted<SR>(cudaStream_t, const Items&, const int2*, const int64_t*,          \
                                               const int64_t*, const DenseWork&, const int64_t*, int64_t*, int32_t*, \
                                               typename SR::T*);
SG_INST(PT64)
SG_INST(MP32)
SG_INST(BOOL8)
SG_INST(PTI64)
#undef SG_INST


// ------------------------------------------------------------------ part sums, colptrs, stats
// nnz of a long column = the sum of its slab counts; spref[s] = rows of the
// column's earlier slabs (where slab s starts inside the column)
__global__ void k_sum_parts(Items it, DenseWork dw, int64_t* __restrict__ nnz_item) {
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= dw.ndense) return;
    const int P = dw.nparts[d];
    const int64_t s0 = dw.sbase[d];
    int32_t acc = 0;
    for (int q = 0; q < P; ++q) {
        dw.spref[s0 + q] = acc;
        acc += dw.scount[s0 + q];
    }
    const int2 e = dw.dlist[d];
    nnz_item[__ldg(it.item_base + e.x) + e.y] = acc;
}

void launch_sum_parts(cudaStream_t st, const Items& it, const DenseWork& dw, int64_t* nnz_item) {
    if (dw.ndense == 0 || dw.dcol) return;   // the dense-column mode counted directly
    k_sum_parts<<<(int)ceil_div64(dw.ndense, 256), 256, 0, st>>>(it, dw, nnz_item);
    note_launch();
}

// colptr_i[j] = offset of the first stored column of B_i with id >= j, relative to the product's start
__global__ void k_colptrs(Items it, const int64_t* __restrict__ colbase, int64_t total, const int64_t* __restrict__ Coff,
                          int64_t* __restrict__ out) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
        int prod = it.nprod == 1 ? 0 : find_prod(colbase, it.nprod, x);
        const Prod* pr = it.prods + prod;
        const int64_t j = x - colbase[prod];
        const int64_t ib = __ldg(it.item_base + prod);
        const int64_t nzc = pr->B.nzc;
        int64_t p;
        if (pr->B.jc == nullptr) {
            p = j;
        } else {
            int64_t lo = 0, hi = nzc;
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if ((int64_t)__ldg(pr->B.jc + mid) < j) lo = mid + 1;
                else hi = mid;
            }
            p = lo;
        }
        out[x] = Coff[ib + p] - Coff[ib];
    }
}

__global__ void k_gather_offsets(const int64_t* __restrict__ Coff, const int64_t* __restrict__ item_base, int64_t np,
                                 int64_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= np; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = Coff[item_base[i]];
}

void launch_gather_offsets(cudaStream_t st, const int64_t* Coff, const int64_t* item_base, int64_t np, int64_t* out) {
    k_gather_offsets<<<(int)ceil_div64(np + 1, 256), 256, 0, st>>>(Coff, item_base, np, out);
    note_launch();
}

void launch_colptrs(cudaStream_t st, const Items& it, const int64_t* colbase, int64_t total_cols, const int64_t* Coff,
                    int64_t* out) {
    if (total_cols <= 0) return;
    int grid = (int)std::min<int64_t>(ceil_div64(total_cols, 256), sm_count() * 16);
    k_colptrs<<<grid, 256, 0, st>>>(it, colbase, total_cols, Coff, out);
    note_launch();
}

__global__ void k_fill_i64(int64_t* p, int64_t n, int64_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

void launch_fill_i64(cudaStream_t st, int64_t* p, int64_t n, int64_t v) {
    if (n <= 0) return;
    int grid = (int)std::min<int64_t>(ceil_div64(n, 256), sm_count() * 16);
    k_fill_i64<<<grid, 256, 0, st>>>(p, n, v);
    note_launch();
}

__global__ void k_tier_stats(Items it, const uint8_t* __restrict__ bin, const int32_t* __restrict__ item_prod,
                             const int64_t* __restrict__ flops, const int64_t* __restrict__ nnz_item,
                             unsigned long long* out) {
    __shared__ unsigned long long s[16];
    if (threadIdx.x < 16) s[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < it.nitems;
         u += (int64_t)gridDim.x * blockDim.x) {
        int b = bin[u];
        int t = b == 0 ? 0 : (b < BIN_BLK0 ? 1 : (b < BIN_DENSE ? 2 : 3));
        int prod = item_prod[u];
        const Prod* pr = it.prods + prod;
        int64_t p = u - __ldg(it.item_base + prod);
        atomicAdd(&s[t], 1ull);
        atomicAdd(&s[4 + t], (unsigned long long)flops[u]);
        atomicAdd(&s[8 + t], (unsigned long long)nnz_item[u]);
        atomicAdd(&s[12 + t], (unsigned long long)(pr->B.cp[p + 1] - pr->B.cp[p]));
    }
    __syncthreads();
    if (threadIdx.x < 16 && s[threadIdx.x]) atomicAdd(out + threadIdx.x, s[threadIdx.x]);
}

void launch_tier_stats(cudaStream_t st, const Items& it, const uint8_t* bin, const int32_t* item_prod,
                       const int64_t* flops, const int64_t* nnz_item, unsigned long long* out) {
    if (it.nitems <= 0) return;
    int grid = (int)std::min<int64_t>(ceil_div64(it.nitems, 256), sm_count() * 4);
    k_tier_stats<<<grid, 256, 0, st>>>(it, bin, item_prod, flops, nnz_item, out);
    note_launch();
}

// ------------------------------------------------------------------ device-wide exclusive scan
constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__device__ __forceinline__ long long block_excl_scan64(long long v, long long* ws, long long& total) {
    long long x = warp_incl_scan64(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        long long s = ws[lane];
        s = warp_incl_scan64(s);
        ws[lane] = s;
    }
    __syncthreads();
    long long add = w > 0 ? ws[w - 1] : 0;
    total = ws[31];
    __syncthreads();
    return x + add - v;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_reduce(const int64_t* __restrict__ in, int64_t n,
                                                             long long* __restrict__ sums) {
    __shared__ long long ws[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    long long s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) s += in[base + i];
    long long total;
    block_excl_scan64(s, ws, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_sums(long long* sums, int64_t nb) {
    __shared__ long long ws[32];
    long long carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_BLOCK) {
        int64_t i = b0 + threadIdx.x;
        long long v = i < nb ? sums[i] : 0;
        long long total;
        long long ex = block_excl_scan64(v, ws, total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_apply(const int64_t* __restrict__ in, int64_t n,
                                                            const long long* __restrict__ sums,
                                                            int64_t* __restrict__ out) {
    __shared__ long long ws[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    long long v[SCAN_ITEMS];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    long long total;
    long long ex = block_excl_scan64(s, ws, total) + sums[blockIdx.x];
    if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        ex += v[i];
        if (base + i < n) out[base + i + 1] = ex;
    }
}

size_t scan_tmp_bytes(int64_t n) { return (size_t)(ceil_div64(std::max<int64_t>(n, 1), SCAN_TILE) + 1) * 8; }

void launch_exclusive_scan(cudaStream_t st, const int64_t* in, int64_t n, int64_t* out, void* tmp) {
    if (n <= 0) {
        cudaMemsetAsync(out, 0, sizeof(int64_t), st);
        return;
    }
    int64_t nb = ceil_div64(n, SCAN_TILE);
    long long* sums = reinterpret_cast<long long*>(tmp);
    k_scan_reduce<<<(int)nb, SCAN_BLOCK, 0, st>>>(in, n, sums);
    k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(sums, nb);
    k_scan_apply<<<(int)nb, SCAN_BLOCK, 0, st>>>(in, n, sums, out);
    note_launch(3);
}

}  // namespace sg
