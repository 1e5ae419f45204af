// Block tier: the numeric pass of every column whose operand A has at most
// BLOCK_TIER_MAX_ROWS rows (the 2D Sparse SUMMA blocks of Section 3.2 and the
// stage merges of Section 6.1 on the virtual grid, and any other short operand).
//
// A group of GS threads (a warp, or a CTA for long columns) takes one output
// column C(:,j) = (+)_{k in B(:,j)} A(:,k) (x) B(k,j) (Section 2.1):
//   1. every product marks its row in a two-level row bitmap in shared memory:
//      L2 holds one bit per row (1024 words for 32768 rows), L1 one bit per
//      nonempty L2 word; lanes that hit the same word combine their bits first;
//   2. one warp turns the bitmap into ranks: per L1 word, the rows before each
//      nonempty L2 word (16-bit) and before the L1 word (int), so the rank of a
//      row is gp + wp + the bits below it in its word;
//   3. C's rows are written at their ranks and C's values set to the semiring zero;
//   4. every product is added into C at its row's rank with an L2 reduction.
// There is no hash table, no sort and no shared-memory accumulator, and the
// bitmap work is proportional to the column's entries, not to the row count.
#include <algorithm>

#include "internal.cuh"

namespace sg {
namespace {

constexpr int L2W = BLOCK_TIER_MAX_ROWS / 32;   // row-bitmap words
constexpr int L1W = L2W / 32;                   // words of the bitmap of nonempty L2 words
static_assert(L1W == 32, "one warp owns the first-level bitmap");

template <class SR, int GS>
struct BtLayout {
    using T = typename SR::T;
    static constexpr size_t l2 = (size_t)L2W * 4;
    static constexpr size_t l1 = (size_t)L1W * 4;
    static constexpr size_t wp = (size_t)L2W * 2;   // rows before each nonempty word (< 2^16)
    static constexpr size_t gp = (size_t)L2W * 2;   // the nonempty words, ascending
    static constexpr size_t incl = (size_t)GS * 4;
    static constexpr size_t a0 = (size_t)GS * 8;
    static constexpr size_t bv = (size_t)GS * 8;
    static constexpr size_t ws = 32 * 8;
    static constexpr size_t group = (l2 + l1 + wp + gp + incl + a0 + bv + ws + 15) / 16 * 16;
};

template <int GS>
__device__ __forceinline__ void gsync() {
    if constexpr (GS == 32) __syncwarp();
    else __syncthreads();
}

// Inclusive scan of a 64-bit value over the group, total in `total`.  For a
// multi-warp group `ws` holds one partial per warp; the closing barrier is left
// to the caller (the next gsync).
template <int GS>
__device__ __forceinline__ long long group_scan64(long long v, long long* ws, long long& total) {
    long long x = warp_incl_scan64(v);
    if constexpr (GS == 32) {
        total = __shfl_sync(0xffffffffu, x, 31);
        return x;
    } else {
        constexpr int NW = GS / 32;
        const int lane = threadIdx.x & 31, w = (threadIdx.x % GS) >> 5;
        if (lane == 31) ws[w] = x;
        __syncthreads();
        if (w == 0) {
            long long s = lane < NW ? ws[lane] : 0;
            s = warp_incl_scan64(s);
            if (lane < NW) ws[lane] = s;
        }
        __syncthreads();
        total = ws[NW - 1];
        return x + (w > 0 ? ws[w - 1] : 0);
    }
}

// Sets bit `bit` of L2 word wd (wd < 0: nothing); the lane that turns a word
// nonzero marks it in L1.  One shared atomic per product: rows of one window
// mostly fall in different words, so folding lanes per word first measured slower.
__device__ __forceinline__ void mark_rows(uint32_t* l2, uint32_t* l1, int wd, uint32_t bit) {
    if (wd < 0) return;
    const uint32_t old = atomicOr(&l2[wd], bit);
    if (old == 0u) atomicOr(&l1[wd >> 5], 1u << (wd & 31));
}

// The products of one chunk of at most GS entries of B(:,j): per entry the
// segment A(:,k), compacted (nonempty segments only); returns the number of
// segments and of products.  Ends with a group barrier.
template <class SR, int GS, bool NUM>
__device__ __forceinline__ void chunk_segments(const Items& it, const Prod* pr, int64_t t, int64_t be, int* s_incl,
                                               int64_t* s_a0, typename SR::T* s_bv, long long* ws, int& ns,
                                               int& total) {
    using T = typename SR::T;
    int len = 0;
    int64_t a0 = 0;
    T bv = T(0);
    if (t < be) {
        const int32_t k = __ldg(pr->B.ir + t);
        int64_t s, e;
        a_col(it, pr, t, k, s, e);
        a0 = s;
        len = (int)(e - s);
        if constexpr (NUM) bv = load_val<SR>(pr->B, t);
    }
    long long tot;
    const long long inc = group_scan64<GS>(len > 0 ? ((1ll << 32) | (unsigned)len) : 0ll, ws, tot);
    if (len > 0) {
        const int p = (int)(inc >> 32) - 1;
        s_incl[p] = (int)(inc & 0xffffffffll);
        s_a0[p] = a0;
        if constexpr (NUM) s_bv[p] = bv;
    }
    ns = (int)(tot >> 32);
    total = (int)(tot & 0xffffffffll);
    gsync<GS>();
}

// Walks the products [0, total) of the current chunk: each warp of the group
// takes a contiguous slice, four 32-product windows per step with every load
// issued first.  f(valid, row, a, b) is called by all 32 lanes of each warp.
template <class SR, int GS, bool NUM, class F>
__device__ __forceinline__ void chunk_walk(const Prod* pr, const int* s_incl, const int64_t* s_a0,
                                           const typename SR::T* s_bv, int ns, int total, F&& f) {
    using T = typename SR::T;
    constexpr int U = 4, NWG = GS / 32;
    const int lane = threadIdx.x & 31, wg = (threadIdx.x % GS) >> 5;
    const int C = (total + NWG * 32 - 1) / (NWG * 32) * 32;
    const int xb = wg * C, xe = min(total, xb + C);
    if (xb >= xe) return;
    int lo = 0, hi = xb > 0 ? ns : 0;   // segments ending at or before the slice start
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_incl[mid] <= xb) lo = mid + 1;
        else hi = mid;
    }
    int o0 = lo;
    const int32_t* __restrict__ air = pr->A.ir;
    int x0 = xb;
    for (; x0 + 32 * (U - 1) < xe; x0 += 32 * U) {   // steps of four full or nearly full windows
        int64_t idx[U];
        bool ok[U];
        int ob[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int xw = x0 + 32 * u;
            const int oi = warp_window_segment(s_incl, ns, xw, o0);
            ok[u] = xw + lane < xe;
            ob[u] = oi;
            idx[u] = ok[u] ? s_a0[oi] + (xw + lane - (oi ? s_incl[oi - 1] : 0)) : 0;
        }
        int32_t row[U];
        T av[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            row[u] = ok[u] ? __ldg(air + idx[u]) : -1;
            if constexpr (NUM) av[u] = ok[u] ? load_val<SR>(pr->A, idx[u]) : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if constexpr (NUM) f(ok[u], row[u], av[u], ok[u] ? s_bv[ob[u]] : T(0));
            else f(ok[u], row[u], T(0), T(0));
        }
    }
    for (; x0 < xe; x0 += 32) {   // the last windows one at a time (short columns end here)
        const int oi = warp_window_segment(s_incl, ns, x0, o0);
        const bool ok = x0 + lane < xe;
        const int64_t idx = ok ? s_a0[oi] + (x0 + lane - (oi ? s_incl[oi - 1] : 0)) : 0;
        const int32_t row = ok ? __ldg(air + idx) : -1;
        if constexpr (NUM) {
            const T av = ok ? load_val<SR>(pr->A, idx) : T(0);
            f(ok, row, av, ok ? s_bv[oi] : T(0));
        } else {
            f(ok, row, T(0), T(0));
        }
    }
}

// Rows of the operand: an out-of-range row (malformed input) is skipped.
__device__ __forceinline__ int row_word(bool ok, int32_t r, int m) { return ok && (unsigned)r < (unsigned)m ? r >> 5 : -1; }

// One column per group.  Coff[u] is where column u starts.  Without nnz_item the
// offsets are exact.  With nnz_item the column's count is recorded there and the
// column is written only when it fits its capacity Coff[u+1] - Coff[u] (the
// predicted and the upper-bound layouts).
// The 512-thread form is held to 32 registers, so that four CTAs (64 warps) stay resident
// per SM: its time is the walk of L2 reductions, which more warps keep in flight.  In the
// FP64 32 x 32 SUMMA at R-MAT scale 20, two CTAs per SM (59 registers) took 3.4 ms longer
// in the stage products and 7.8 ms longer in the merge; three CTAs took 0.4 and 2.0 ms longer.
template <class SR, int GS, int BLOCK>
__global__ void __launch_bounds__(BLOCK, BLOCK == 512 ? 4 : 1) k_block_tier(Items it, const int2* __restrict__ list, int64_t count,
                                                     int64_t* __restrict__ nnz_item, const int64_t* __restrict__ Coff,
                                                     int32_t* __restrict__ Cir, typename SR::T* __restrict__ Cv,
                                                     const int* __restrict__ vals_zero) {
    using T = typename SR::T;
    using L = BtLayout<SR, GS>;
    constexpr int NG = BLOCK / GS;
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = (threadIdx.x / GS), lane = threadIdx.x % GS;
    unsigned char* base = smem + (size_t)g * L::group;
    uint32_t* l2 = reinterpret_cast<uint32_t*>(base);
    uint32_t* l1 = reinterpret_cast<uint32_t*>(base + L::l2);
    uint16_t* wp = reinterpret_cast<uint16_t*>(base + L::l2 + L::l1);
    uint16_t* wl = reinterpret_cast<uint16_t*>(base + L::l2 + L::l1 + L::wp);
    int* s_incl = reinterpret_cast<int*>(base + L::l2 + L::l1 + L::wp + L::gp);
    int64_t* s_a0 = reinterpret_cast<int64_t*>(base + L::l2 + L::l1 + L::wp + L::gp + L::incl);
    T* s_bv = reinterpret_cast<T*>(base + L::l2 + L::l1 + L::wp + L::gp + L::incl + L::a0);
    long long* ws = reinterpret_cast<long long*>(base + L::l2 + L::l1 + L::wp + L::gp + L::incl + L::a0 + L::bv);
    // boolean products whose operands hold no false value: every output value is true
    const bool walk = SR::id != SPGEMM_OR_AND_BOOL || vals_zero == nullptr || *vals_zero != 0;
    const T init = walk ? SR::out(SR::zero()) : T(1);
    for (int x = lane; x < L2W; x += GS) l2[x] = 0u;
    for (int x = lane; x < L1W; x += GS) l1[x] = 0u;
    gsync<GS>();
    for (int64_t w = (int64_t)blockIdx.x * NG + g; w < count; w += (int64_t)gridDim.x * NG) {
        const int2 e = __ldg(list + w);
        const Prod* pr = it.prods + e.x;
        const int64_t u = __ldg(it.item_base + e.x) + e.y;
        const int64_t bs = __ldg(pr->B.cp + e.y), be = __ldg(pr->B.cp + e.y + 1);
        const int m = (int)pr->A.m;   // <= BLOCK_TIER_MAX_ROWS
        const int nw = (m + 31) >> 5;
        const bool one_chunk = be - bs <= GS;
        int ns = 0, total = 0;
        // 1. marks
        for (int64_t b0 = bs; b0 < be; b0 += GS) {
            // the B values too: a single chunk's segments serve the value pass as they are
            chunk_segments<SR, GS, true>(it, pr, b0 + lane, be, s_incl, s_a0, s_bv, ws, ns, total);
            chunk_walk<SR, GS, false>(pr, s_incl, s_a0, s_bv, ns, total, [&](bool ok, int32_t r, T, T) {
                mark_rows(l2, l1, row_word(ok, r, m), 1u << (r & 31));
            });
            if (!one_chunk) gsync<GS>();   // the next chunk rewrites the segment arrays
        }
        gsync<GS>();
        // 2. ranks, by warp 0 of the group: the nonempty words in ascending order (from L1,
        //    by a warp scan of the per-word counts), then the rows before each of them
        //    (32 words per step).  A row's rank is wp[its word] + the bits below it there.
        if (lane < 32) {
            const uint32_t lb = l1[lane];
            const int nl = __popc(lb);
            const int off = warp_incl_scan(nl) - nl;
            const int nwords = __shfl_sync(0xffffffffu, off + nl, 31);
            uint32_t bits = lb;
            for (int i = 0; bits; ++i) {   // lane l lists the words of L1 word l
                wl[off + i] = (uint16_t)(lane * 32 + __ffs(bits) - 1);
                bits &= bits - 1;
            }
            __syncwarp();
            int carry = 0;
            for (int i0 = 0; i0 < nwords; i0 += 32) {
                const int i = i0 + lane;
                const int wd = i < nwords ? wl[i] : 0;
                const int c = i < nwords ? __popc(l2[wd]) : 0;
                const int incl = warp_incl_scan(c);
                if (i < nwords) wp[wd] = (uint16_t)(carry + incl - c);
                carry += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) {
                ws[0] = carry;    // the column's entries
                ws[1] = nwords;   // its nonempty words
            }
        }
        gsync<GS>();
        const int cnt = (int)ws[0];
        const int nwords = (int)ws[1];
        const int64_t out0 = __ldg(Coff + u);
        const int64_t capn = __ldg(Coff + u + 1) - out0;
        // exact offsets always fit (the counting pass marks the same rows); the check
        // keeps an inconsistent input from writing past the column
        const bool write = cnt <= capn;
        if (nnz_item && lane == 0) nnz_item[u] = cnt;
        const int32_t rb = out_row_base(pr, e.y);
        if (write) {
            // 3. rows at their ranks (evict-first: written once), values set to the semiring
            //    zero (kept in L2 for the reductions that follow).  Each warp of the group
            //    takes 32 nonempty words at a time: one word per lane, bit by bit, when the
            //    words are sparse; word by word with the whole warp (one coalesced store per
            //    word) when they are dense.
            {
                const int wlane = threadIdx.x & 31, wgi = (threadIdx.x % GS) >> 5;
                for (int i0 = wgi * 32; i0 < nwords; i0 += GS) {
                    const int i = i0 + wlane;
                    const int wd = i < nwords ? wl[i] : 0;
                    uint32_t wv = i < nwords ? l2[wd] : 0u;
                    const int r0 = i < nwords ? wp[wd] : 0;
                    const int pc = __popc(wv);
                    if (__reduce_add_sync(0xffffffffu, pc) >= 16 * 32) {
                        for (int j = 0; j < 32; ++j) {
                            const int wdj = __shfl_sync(0xffffffffu, wd, j);
                            const uint32_t wvj = __shfl_sync(0xffffffffu, wv, j);
                            const int rj = __shfl_sync(0xffffffffu, r0, j);
                            if (i0 + j < nwords && ((wvj >> wlane) & 1u))
                                __stcs(Cir + out0 + rj + __popc(wvj & ((1u << wlane) - 1u)), wdj * 32 + wlane + rb);
                        }
                    } else {
                        int r = r0;
                        while (wv) {
                            __stcs(Cir + out0 + r++, wd * 32 + __ffs(wv) - 1 + rb);
                            wv &= wv - 1;
                        }
                    }
                }
            }
            for (int i = lane; i < cnt; i += GS) Cv[out0 + i] = init;
            gsync<GS>();   // this group's stores come before its reductions
            // 4. every product added at its row's rank
            if (walk) {
                for (int64_t b0 = bs; b0 < be; b0 += GS) {
                    if (!one_chunk) chunk_segments<SR, GS, true>(it, pr, b0 + lane, be, s_incl, s_a0, s_bv, ws, ns, total);
                    chunk_walk<SR, GS, true>(pr, s_incl, s_a0, s_bv, ns, total, [&](bool ok, int32_t r, T a, T b) {
                        if (!ok || (unsigned)r >= (unsigned)m) return;
                        const int wd = r >> 5;
                        const uint32_t wv = l2[wd];
                        const uint32_t bit = 1u << (r & 31);
                        const int rank = wp[wd] + __popc(wv & (bit - 1u));
                        red_out<SR>(Cv, out0 + rank, SR::mul(a, b));
                    });
                    if (!one_chunk) gsync<GS>();
                }
            }
        }
        gsync<GS>();
        // 5. clear the touched words (through the word list)
        for (int i = lane; i < nwords; i += GS) l2[wl[i]] = 0u;
        if (lane < L1W) l1[lane] = 0u;
        gsync<GS>();
    }
}

// ------------------------------------------------------------------ sort tier
// Columns of at most N = 32 K products (bins 2, 3 and 4 when the tier configuration
// bounds their flops, K = 1, 2 and 4), one warp each, in registers: slot i = 32 r + lane
// receives product i keyed (row << 7) | i, a bitonic network across the warp sorts
// the keys (the values follow through the slot index), a segmented scan combines
// equal rows, and C's rows and values are written with coalesced stores.  There is
// no bitmap to set up and clear, no shared memory and no atomic, which is what
// dominates the block tier's cost on columns this short.

// A lane's register shuffled up by d lanes, or from lane src (one-byte types through int).
template <class V>
__device__ __forceinline__ V shfl_v_up(V x, int d) {
    if constexpr (sizeof(V) == 1) return (V)__shfl_up_sync(0xffffffffu, (int)x, d);
    else return __shfl_up_sync(0xffffffffu, x, d);
}

template <class V>
__device__ __forceinline__ V shfl_v(V x, int src) {
    if constexpr (sizeof(V) == 1) return (V)__shfl_sync(0xffffffffu, (int)x, src);
    else return __shfl_sync(0xffffffffu, x, src);
}

template <class SR, int K>
__global__ void __launch_bounds__(256) k_sort_tier(Items it, const int2* __restrict__ list, int64_t count,
                                                   int64_t* __restrict__ nnz_item, const int64_t* __restrict__ Coff,
                                                   int32_t* __restrict__ Cir, typename SR::T* __restrict__ Cv,
                                                   const int* __restrict__ vals_zero) {
    using T = typename SR::T;
    using Acc = typename SR::Acc;
    constexpr int N = 32 * K;
    constexpr uint32_t NONE = 0xffffffffu;
    static_assert(K == 1 || K == 2 || K == 4, "slot index fits 7 bits; rows fit 25 bits");
    const int lane = threadIdx.x & 31;
    // boolean products whose operands hold no false value: every output value is true
    const bool walk = SR::id != SPGEMM_OR_AND_BOOL || vals_zero == nullptr || *vals_zero != 0;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < count; w += nwarp) {
        const int2 e = __ldg(list + w);
        const Prod* pr = it.prods + e.x;
        const int64_t u = __ldg(it.item_base + e.x) + e.y;
        const int64_t bs = __ldg(pr->B.cp + e.y), be = __ldg(pr->B.cp + e.y + 1);
        const int m = (int)pr->A.m;   // <= BLOCK_TIER_MAX_ROWS
        uint32_t key[K];
        Acc val[K];
#pragma unroll
        for (int r = 0; r < K; ++r) {
            key[r] = NONE;
            val[r] = SR::zero();
        }
        // 1. products into slots: the entries of B(:,j) 32 at a time, slot i holding
        //    product i (the bin bounds the column's products by N)
        int base = 0;
        for (int64_t b0 = bs; b0 < be && base < N; b0 += 32) {
            const int64_t t = b0 + lane;
            int len = 0;
            int64_t a0 = 0;
            T bv = T(0);
            if (t < be) {
                const int32_t k = __ldg(pr->B.ir + t);
                int64_t sa, ea;
                a_col(it, pr, t, k, sa, ea);
                a0 = sa;
                len = (int)(ea - sa);
                if (walk) bv = load_val<SR>(pr->B, t);
            }
            const int inc = warp_incl_scan(len);
            const int tot = __shfl_sync(0xffffffffu, inc, 31);
#pragma unroll
            for (int r = 0; r < K; ++r) {
                const int p = r * 32 + lane - base;   // the slot's product within this chunk
                int src = 0;                          // entries that end at or before product p
#pragma unroll
                for (int st = 16; st > 0; st >>= 1)
                    if (__shfl_sync(0xffffffffu, inc, src + st - 1) <= p) src += st;
                const int ex = __shfl_sync(0xffffffffu, inc - len, src);
                const int64_t as = __shfl_sync(0xffffffffu, a0, src);
                const T bvs = shfl_v(bv, src);
                if (p >= 0 && p < tot) {
                    const int64_t pos = as + (p - ex);
                    const int32_t row = __ldg(pr->A.ir + pos);
                    if ((unsigned)row < (unsigned)m) {   // else malformed input: skipped
                        key[r] = ((uint32_t)row << 7) | (uint32_t)(r * 32 + lane);
                        val[r] = walk ? SR::mul(load_val<SR>(pr->A, pos), bvs) : SR::one();
                    }
                }
            }
            base += tot;
        }
        // 2. bitonic sort of the N keys (slot i = 32 r + lane; partner i ^ j)
#pragma unroll
        for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                uint32_t nk[K];
#pragma unroll
                for (int r = 0; r < K; ++r) {
                    const int i = r * 32 + lane;
                    const uint32_t kp = j >= 32 ? key[r ^ (j >> 5)] : __shfl_xor_sync(0xffffffffu, key[r], j);
                    const bool take_min = ((i & k) == 0) == ((i & j) == 0);
                    nk[r] = take_min ? min(key[r], kp) : max(key[r], kp);
                }
#pragma unroll
                for (int r = 0; r < K; ++r) key[r] = nk[r];
            }
        }
        // 3. every sorted key takes its slot's value; equal rows are combined by a
        //    segmented scan (equal rows are adjacent), so a row's last slot holds its sum
        Acc v[K];
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const int idx = (int)(key[r] & 127u);
            Acc x = shfl_v(val[0], idx & 31);
#pragma unroll
            for (int q = 1; q < K; ++q) {
                const Acc y = shfl_v(val[q], idx & 31);
                x = (idx >> 5) == q ? y : x;
            }
            v[r] = x;
        }
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const uint32_t rw = key[r] >> 7;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t rp = __shfl_up_sync(0xffffffffu, rw, d);
                const Acc vp = shfl_v_up(v[r], d);
                if (lane >= d && rp == rw) v[r] = SR::add(vp, v[r]);
            }
        }
#pragma unroll
        for (int r = 1; r < K; ++r) {   // a row whose slots continue from register r - 1 into r
            const uint32_t cr = __shfl_sync(0xffffffffu, key[r - 1] >> 7, 31);
            const Acc cv = shfl_v(v[r - 1], 31);
            if (key[r] != NONE && (key[r] >> 7) == cr) v[r] = SR::add(cv, v[r]);
        }
        // 4. a row's last slot writes it: positions by ballots, coalesced stores
        uint32_t tb[K];
        int cnt = 0;
#pragma unroll
        for (int r = 0; r < K; ++r) {
            const uint32_t rw = key[r] >> 7;
            uint32_t nx = __shfl_down_sync(0xffffffffu, rw, 1);
            const uint32_t first_next = __shfl_sync(0xffffffffu, key[r + 1 < K ? r + 1 : r] >> 7, 0);
            if (lane == 31) nx = r + 1 < K ? first_next : NONE;
            tb[r] = __ballot_sync(0xffffffffu, key[r] != NONE && nx != rw);
            cnt += __popc(tb[r]);
        }
        const int64_t out0 = __ldg(Coff + u);
        const int64_t capn = __ldg(Coff + u + 1) - out0;
        if (nnz_item && lane == 0) nnz_item[u] = cnt;
        // exact offsets always fit; with nnz_item a column that does not fit its slots
        // is only counted
        if (cnt <= capn) {
            const int32_t rb = out_row_base(pr, e.y);
            int before = 0;
#pragma unroll
            for (int r = 0; r < K; ++r) {
                if ((tb[r] >> lane) & 1u) {
                    const int pos = before + __popc(tb[r] & ((1u << lane) - 1u));
                    __stcs(Cir + out0 + pos, (int32_t)(key[r] >> 7) + rb);
                    Cv[out0 + pos] = SR::out(v[r]);
                }
                before += __popc(tb[r]);
            }
        }
    }
}

template <class SR, int K>
void run_sort(cudaStream_t st, const Items& it, const int2* list, int64_t count, int64_t* nnz_item,
              const int64_t* Coff, int32_t* Cir, typename SR::T* Cv, const int* vals_zero) {
    if (count <= 0) return;
    const int grid = (int)std::min<int64_t>(ceil_div64(count, 8), (int64_t)sm_count() * 8);
    k_sort_tier<SR, K><<<grid, 256, 0, st>>>(it, list, count, nnz_item, Coff, Cir, Cv, vals_zero);
    note_launch();
}

template <class SR, int GS, int BLOCK>
void run_bt(cudaStream_t st, const Items& it, const int2* list, int64_t count, int64_t* nnz_item, const int64_t* Coff,
            int32_t* Cir, typename SR::T* Cv, const int* vals_zero) {
    if (count <= 0) return;
    constexpr int NG = BLOCK / GS;
    const size_t smem = BtLayout<SR, GS>::group * NG;
    auto kern = k_block_tier<SR, GS, BLOCK>;
    static bool attr = false;   // per process: the limit belongs to the kernel
    if (!attr) {
        cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int grid = (int)std::min<int64_t>(ceil_div64(count, NG), (int64_t)per_sm * sm_count());
    kern<<<grid, BLOCK, smem, st>>>(it, list, count, nnz_item, Coff, Cir, Cv, vals_zero);
    note_launch();
}

}  // namespace

template <class SR>
void launch_block_tier(cudaStream_t st, const Items& it, const int2* list, const int64_t* bin_off,
                       const int64_t* bin_cnt, const DenseWork& dw, int64_t* nnz_item, const int64_t* Coff,
                       int32_t* Cir, typename SR::T* Cv, int which) {
    if (which & 1) {
        // Bins [b0, b1) as one launch per contiguous run: the lists of the exact and
        // predicted passes are contiguous, but a repair list keeps every bin at its
        // full-list offset with fewer entries, which leaves gaps between bins.
        auto runs = [&](int b0, int b1, auto launch) {
            int b = b0;
            while (b < b1) {
                const int64_t start = bin_off[b];
                int64_t n = 0;
                int e = b;
                while (e < b1 && bin_off[e] == start + n) n += bin_cnt[e++];
                if (e == b) {   // bin b starts after a gap: a run of its own
                    n = bin_cnt[b];
                    e = b + 1;
                }
                launch(list + start, n);
                b = e;
            }
        };
        // bins 2, 3 and 4 (at most 32, 64 and 128 products per column here): the sort tier
        run_sort<SR, 1>(st, it, list + bin_off[BIN_WARP0], bin_cnt[BIN_WARP0], nnz_item, Coff, Cir, Cv,
                        dw.vals_zero);
        run_sort<SR, 2>(st, it, list + bin_off[BIN_WARP0 + 1], bin_cnt[BIN_WARP0 + 1], nnz_item, Coff, Cir, Cv,
                        dw.vals_zero);
        run_sort<SR, 4>(st, it, list + bin_off[BIN_WARP0 + 2], bin_cnt[BIN_WARP0 + 2], nnz_item, Coff, Cir, Cv,
                        dw.vals_zero);
        // one warp per column for the other warp bins and the CTA-table bins too (cap <=
        // 4096): without the CTA's barrier chain per column, measured faster than
        // 256-thread groups
        runs(BIN_WARP0 + 3, BIN_DENSE, [&](const int2* l, int64_t n) {
            run_bt<SR, 32, 256>(st, it, l, n, nnz_item, Coff, Cir, Cv, dw.vals_zero);
        });
    }
    // long columns (cap > 4096): a 512-thread group each (one warp each measured slower)
    if (which & 2) run_bt<SR, 512, 512>(st, it, dw.dlist, dw.ndense, nnz_item, Coff, Cir, Cv, dw.vals_zero);
}

#define SG_INST(SR)                                                                                               \
    template void launch_block_tier<SR>(cudaStream_t, const Items&, const int2*, const int64_t*, const int64_t*, \
                                        const DenseWork&, int64_t*, const int64_t*, int32_t*, typename SR::T*, int);
SG_INST(PT64)
SG_INST(MP32)
SG_INST(BOOL8)
SG_INST(PTI64)
#undef SG_INST

}  // namespace sg
