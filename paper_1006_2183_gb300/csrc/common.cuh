// Shared device-side definitions of the SpGEMM library: semiring traits,
// matrix views (CSC / DCSC with AUX), and thread-group primitives.
#pragma once
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "spgemm.h"

namespace sg {

// ------------------------------------------------------------------ semirings
// Each semiring gives the stored element type T, the shared-memory
// accumulator type Acc (wide enough for a native shared atomic), the additive
// identity, (x), and an atomic (+) on a shared accumulator (Section 1: SpGEMM
// over an arbitrary semiring).
struct PT64 {
    using T = double;
    using Acc = double;
    static constexpr int id = SPGEMM_PLUS_TIMES_F64;
    __device__ static Acc zero() { return 0.0; }
    __device__ static Acc one() { return 1.0; }
    __device__ static Acc mul(T a, T b) { return __dmul_rn(a, b); }
    __device__ static Acc add(Acc a, Acc b) { return __dadd_rn(a, b); }
    __device__ static void atomic_add(Acc* p, Acc x) { atomicAdd(p, x); }
    __device__ static T out(Acc a) { return a; }
};

struct MP32 {
    using T = float;
    using Acc = float;
    static constexpr int id = SPGEMM_MIN_PLUS_F32;
    __device__ static Acc zero() { return CUDART_INF_F; }
    __device__ static Acc one() { return 0.0f; }
    __device__ static Acc mul(T a, T b) { return __fadd_rn(a, b); }
    __device__ static Acc add(Acc a, Acc b) { return b < a ? b : a; }
    // min on floats through integer atomics: for x >= 0 the IEEE bit patterns
    // order like signed ints; for x < 0 they order in reverse as unsigned ints.
    __device__ static void atomic_add(Acc* p, Acc x) {
        if (x >= 0.0f) atomicMin(reinterpret_cast<int*>(p), __float_as_int(x));
        else atomicMax(reinterpret_cast<unsigned int*>(p), __float_as_uint(x));
    }
    __device__ static T out(Acc a) { return a; }
};

struct BOOL8 {
    using T = uint8_t;
    using Acc = unsigned int;
    static constexpr int id = SPGEMM_OR_AND_BOOL;
    __device__ static Acc zero() { return 0u; }
    __device__ static Acc one() { return 1u; }
    __device__ static Acc mul(T a, T b) { return (a != 0 && b != 0) ? 1u : 0u; }
    __device__ static Acc add(Acc a, Acc b) { return a | b; }
    __device__ static void atomic_add(Acc* p, Acc x) { if (x) atomicOr(p, x); }
    __device__ static T out(Acc a) { return (T)(a != 0); }
};

struct PTI64 {
    using T = int64_t;
    using Acc = unsigned long long;
    static constexpr int id = SPGEMM_PLUS_TIMES_I64;
    __device__ static Acc zero() { return 0ull; }
    __device__ static Acc one() { return 1ull; }
    __device__ static Acc mul(T a, T b) { return (Acc)a * (Acc)b; }
    __device__ static Acc add(Acc a, Acc b) { return a + b; }
    __device__ static void atomic_add(Acc* p, Acc x) { atomicAdd(p, x); }
    __device__ static T out(Acc a) { return (T)a; }
};

// ------------------------------------------------------------------ matrix view
// CSC when jc == nullptr; DCSC (Section 2.3) otherwise: cp[p], jc[p] describe the
// p-th nonempty column, aux indexes chunks of `chunk` columns.
struct DMat {
    int64_t m = 0, n = 0;     // rows, columns (full dimensions)
    int64_t nzc = 0;          // stored columns (n for CSC)
    int64_t nnz = 0;
    const int64_t* cp = nullptr;
    const int32_t* jc = nullptr;
    const int32_t* aux = nullptr;
    int64_t chunk = 1, naux = 0;
    const int32_t* ir = nullptr;
    const void* num = nullptr;  // nullptr: pattern only (values = semiring one)
    const int64_t* ce = nullptr;  // CSC with gaps: column k holds [cp[k], ce[k]) (else [cp[k], cp[k+1]))
};

// One product of a batch.  Its items are the stored columns p of B; item p has
// the global index item_base + p.  Output rows are written shifted by row_base.
struct Prod {
    DMat A, B;
    int64_t item_base = 0;   // first global item of this product
    int64_t bnz_base = 0;    // sum of nnz(B) over earlier products (cursor addressing)
    int32_t row_base = 0;    // added to every output row id
    int64_t col_base = 0;    // global column of B's column 0 (2D blocks)
    int32_t tag = 0;         // caller's label (SUMMA: the stage)
    int32_t blk = 0;         // caller's second label (SUMMA: the block row)
    int32_t rb_cycle = 0;    // > 0: item p's rows also get (p mod rb_cycle) * rb_step
    int32_t rb_step = 0;
};

// Offset added to the output rows of column p of a product: row_base, plus
// (p mod rb_cycle) * rb_step when B's columns interleave row blocks (the SUMMA
// merge numbers its output columns j * g + I for row block I).
__device__ __forceinline__ int32_t out_row_base(const Prod* pr, int64_t p) {
    const int32_t c = pr->rb_cycle;
    return pr->row_base + (c > 0 ? (int32_t)(p % c) * pr->rb_step : 0);
}

template <class SR>
__device__ __forceinline__ typename SR::T load_val(const DMat& M, int64_t idx) {
    if (M.num == nullptr) return (typename SR::T)SR::one();
    return __ldg(reinterpret_cast<const typename SR::T*>(M.num) + idx);
}

// Column k of A as a half-open range of positions; empty -> s == e.
// DCSC: chunk t = k / chunk holds JC positions [aux[t], aux[t+1]) (AUX, Section 2.3).
__device__ __forceinline__ void col_range(const DMat& A, int32_t k, int64_t& s, int64_t& e) {
    if (k < 0 || (int64_t)k >= A.n) {   // malformed operand: treat as an empty column
        s = e = 0;
        return;
    }
    if (A.jc == nullptr) {
        s = __ldg(A.cp + k);
        e = A.ce ? __ldg(A.ce + k) : __ldg(A.cp + k + 1);
        return;
    }
    const int64_t t = (uint32_t)k / (uint32_t)A.chunk;   // 0 <= k < n < 2^31 and 1 <= chunk <= n
    int32_t p0 = __ldg(A.aux + t), p1 = __ldg(A.aux + t + 1);
    for (int32_t p = p0; p < p1; ++p) {
        int32_t c = __ldg(A.jc + p);
        if (c == k) { s = __ldg(A.cp + p); e = __ldg(A.cp + p + 1); return; }
        if (c > k) break;
    }
    s = e = 0;
}

// col_range for two columns at once (k < 0 or >= n: an empty column), each level of
// the lookups issued for both before the next: AUX, the first JC candidate, CP.  (Four
// at once measured slower: more registers, fewer warps per SM.)
__device__ __forceinline__ void col_range2(const DMat& A, const int32_t (&k)[2], int64_t (&s)[2], int64_t (&e)[2]) {
    bool ok[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) ok[i] = k[i] >= 0 && (int64_t)k[i] < A.n;
    if (A.jc == nullptr) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            s[i] = ok[i] ? __ldg(A.cp + k[i]) : 0;
            e[i] = ok[i] ? (A.ce ? __ldg(A.ce + k[i]) : __ldg(A.cp + k[i] + 1)) : 0;
        }
        return;
    }
    int32_t p0[2], p1[2], c[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int64_t t = ok[i] ? (uint32_t)k[i] / (uint32_t)A.chunk : 0;   // 0 <= k < n < 2^31
        p0[i] = ok[i] ? __ldg(A.aux + t) : 0;
        p1[i] = ok[i] ? __ldg(A.aux + t + 1) : 0;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) c[i] = p0[i] < p1[i] ? __ldg(A.jc + p0[i]) : INT_MAX;
#pragma unroll
    for (int i = 0; i < 2; ++i)
        while (c[i] < k[i]) {   // later columns of the same AUX chunk (rare)
            ++p0[i];
            c[i] = p0[i] < p1[i] ? __ldg(A.jc + p0[i]) : INT_MAX;
        }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hit = ok[i] && c[i] == k[i];
        s[i] = hit ? __ldg(A.cp + p0[i]) : 0;
        e[i] = hit ? __ldg(A.cp + p0[i] + 1) : 0;
    }
}

__device__ __forceinline__ int64_t col_len(const DMat& A, int32_t k) {
    int64_t s, e;
    col_range(A, k, s, e);
    return e - s;
}

// ------------------------------------------------------------------ group helpers
// A "group" of GS threads cooperates on one output column: GS == 32 is a warp,
// GS == blockDim.x is the whole CTA.
template <int GS>
struct Group {
    static_assert(GS == 32 || GS % 32 == 0, "group size");
    __device__ static int lane() { return threadIdx.x % GS; }
    __device__ static int gid() { return threadIdx.x / GS; }
    __device__ static void sync() {
        if constexpr (GS == 32) __syncwarp();
        else __syncthreads();
    }
};

__device__ __forceinline__ int warp_incl_scan(int v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ long long warp_incl_scan64(long long v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Inclusive scan over a group of GS threads (GS a multiple of 32), through
// `scratch` (GS/32 ints).  Also returns the group total.
template <int GS>
__device__ __forceinline__ int group_incl_scan(int v, int* scratch, int& total) {
    int x = warp_incl_scan(v);
    if constexpr (GS == 32) {
        total = __shfl_sync(0xffffffffu, x, 31);
        return x;
    } else {
        constexpr int NW = GS / 32;
        int lane = threadIdx.x & 31, w = (threadIdx.x % GS) >> 5;
        if (lane == 31) scratch[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = lane < NW ? scratch[lane] : 0;
            s = warp_incl_scan(s);
            if (lane < NW) scratch[lane] = s;
        }
        __syncthreads();
        int add = w > 0 ? scratch[w - 1] : 0;
        total = scratch[NW - 1];
        __syncthreads();
        return x + add;
    }
}

// group_incl_scan without its closing barrier: the caller must reach another
// barrier of the group (or, for a warp, a full-warp shuffle) before the next call
// writes `scratch` again.
template <int GS>
__device__ __forceinline__ int group_incl_scan_open(int v, int* scratch, int& total) {
    int x = warp_incl_scan(v);
    if constexpr (GS == 32) {
        total = __shfl_sync(0xffffffffu, x, 31);
        return x;
    } else {
        constexpr int NW = GS / 32;
        int lane = threadIdx.x & 31, w = (threadIdx.x % GS) >> 5;
        if (lane == 31) scratch[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = lane < NW ? scratch[lane] : 0;
            s = warp_incl_scan(s);
            if (lane < NW) scratch[lane] = s;
        }
        __syncthreads();
        total = scratch[NW - 1];
        return x + (w > 0 ? scratch[w - 1] : 0);
    }
}

// 64-bit group_incl_scan_open for a group of several warps (GS == blockDim.x),
// scratch of GS / 32 entries.
template <int GS>
__device__ __forceinline__ long long group_incl_scan64_open(long long v, long long* scratch, long long& total) {
    static_assert(GS > 32 && GS % 32 == 0, "several warps");
    constexpr int NW = GS / 32;
    const int lane = threadIdx.x & 31, w = (threadIdx.x % GS) >> 5;
    long long x = warp_incl_scan64(v);
    if (lane == 31) scratch[w] = x;
    __syncthreads();
    if (w == 0) {
        long long s = lane < NW ? scratch[lane] : 0;
        s = warp_incl_scan64(s);
        if (lane < NW) scratch[lane] = s;
    }
    __syncthreads();
    total = scratch[NW - 1];
    return x + (w > 0 ? scratch[w - 1] : 0);
}

// Segment of product xw + lane for a warp over compacted segments (ends[0, ns)
// strictly increasing: no empty segment): bit b of the window mask marks the
// segment that ends at xw + b + 1, so the lane's segment index is the count of
// segments ending at or before its product.  o0 carries the segments that end at
// or before the window start; windows must come in order.  All 32 lanes call it.
__device__ __forceinline__ int warp_window_segment(const int* ends, int ns, int xw, int& o0) {
    const int lane = threadIdx.x & 31;
    const int ej = o0 + lane < ns ? ends[o0 + lane] : INT_MAX;
    const unsigned bitv = (ej > xw && ej <= xw + 32) ? (1u << (ej - xw - 1)) : 0u;
    const unsigned mask = __reduce_or_sync(0xffffffffu, bitv);
    const int oi = o0 + __popc(mask & ((1u << lane) - 1u));
    o0 += __popc(mask);
    return oi;
}

// Asynchronous 16-byte copy global -> shared (both 16-byte aligned), completed by
// cp_async_wait_all in the issuing thread (then a barrier publishes it).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// C[pos] = C[pos] (+) v in global memory (an L2 reduction; the return value is unused).
template <class SR>
__device__ __forceinline__ void red_out(typename SR::T* Cv, int64_t pos, typename SR::Acc v) {
    if constexpr (SR::id == SPGEMM_OR_AND_BOOL) {
        if (v) {
            const uintptr_t a = reinterpret_cast<uintptr_t>(Cv + pos);
            atomicOr(reinterpret_cast<unsigned int*>(a & ~uintptr_t(3)), 1u << ((a & 3) * 8));
        }
    } else if constexpr (SR::id == SPGEMM_PLUS_TIMES_I64) {
        atomicAdd(reinterpret_cast<unsigned long long*>(Cv + pos), v);
    } else {
        SR::atomic_add(Cv + pos, v);   // double add; float min through integer min / max
    }
}

// bitmap[wd] |= bit for every lane with wd >= 0; lanes that hit the same word
// combine their bits first, so each run of equal words takes one shared atomic.
// Called by all 32 lanes of the warp.
__device__ __forceinline__ void or_bits_warp(uint32_t* bitmap, int wd, uint32_t bit) {
    const int lane = threadIdx.x & 31;
    const int wprev = __shfl_up_sync(0xffffffffu, wd, 1);
    const bool head = lane == 0 || wprev != wd;
    uint32_t acc = bit;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t b2 = __shfl_down_sync(0xffffffffu, acc, o);
        const int w2 = __shfl_down_sync(0xffffffffu, wd, o);
        if (lane + o < 32 && w2 == wd) acc |= b2;
    }
    if (wd >= 0 && head) atomicOr(&bitmap[wd], acc);
}

__host__ __device__ __forceinline__ int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ uint32_t hash_row(int32_t r) { return (uint32_t)r * 0x9E3779B1u; }

}  // namespace sg
