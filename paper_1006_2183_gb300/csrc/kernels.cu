// Flat column-wise SpGEMM kernels (Gustavson's column-by-column formulation,
// Section 2.1; accumulation in the spirit of the sparse accumulator of
// Section 3.3), organised in three accumulator tiers chosen per output column
// from cap_j = min(flops_j, m):
//   * warp-wide shared-memory hash tables (short columns),
//   * CTA-wide shared-memory hash tables (medium columns),
//   * a row-chunked dense accumulator (long columns): R rows of values plus an
//     R-bit occupancy map per chunk, walked chunk by chunk with per-(column,k)
//     cursors into A(:,k); rows come out sorted, so no sort is needed.
// The symbolic pass counts nnz(C(:,j)); the numeric pass fills rows and values.
#include <algorithm>
#include <climits>

#include <atomic>

#include "kernels.cuh"

namespace sg {

static std::atomic<int64_t> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launches() { return g_launches.load(std::memory_order_relaxed); }

constexpr int WARP_BLOCK = 256;   // 8 warp groups per CTA
constexpr int DENSE_BLOCK = 512;

__host__ __device__ __forceinline__ int bin_of(int64_t cap, int warp_max, int block_max) {
    if (cap <= 0) return 0;
    if (cap <= warp_max) {
        int64_t t = WARP_TBL0;
        int b = 1;
        while (t < 2 * cap) { t <<= 1; ++b; }
        return b;
    }
    if (cap <= block_max) {
        int64_t t = BLK_TBL0;
        int b = 1 + NWARP;
        while (t < 2 * cap) { t <<= 1; ++b; }
        return b;
    }
    return BIN_DENSE;
}

int dense_rows_for(int semiring, int requested) {
    if (requested > 0) return std::max(32, (requested / 32) * 32);
    switch (semiring) {
    case SPGEMM_PLUS_TIMES_F64:
    case SPGEMM_PLUS_TIMES_I64: return 8192;
    default: return 16384;
    }
}

// ------------------------------------------------------------------ analysis
// Groups of 8 lanes per stored column of B: flops_j = sum_k nnz(A(:,k))
// (Section 1), the tier bin, and optionally the predictor inputs.
__global__ void __launch_bounds__(256) k_analyze(DMat A, DMat B, TierCfg cfg, int64_t* __restrict__ flops,
                                                 uint8_t* __restrict__ bin, unsigned long long* bin_count,
                                                 unsigned long long* flops_total, const uint64_t* __restrict__ sketch,
                                                 float* __restrict__ feat) {
    __shared__ unsigned long long s_cnt[NBIN];
    __shared__ unsigned long long s_fl;
    if (threadIdx.x < NBIN) s_cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_fl = 0;
    __syncthreads();
    const int sub = threadIdx.x & 7;
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    long long f = 0;
    long long mx = 0;
    unsigned long long sk = 0;
    int64_t bs = 0, be = 0;
    if (p < B.nzc) {
        bs = __ldg(B.cp + p);
        be = __ldg(B.cp + p + 1);
        for (int64_t t = bs + sub; t < be; t += 8) {
            int32_t k = __ldg(B.ir + t);
            long long len = col_len(A, k);
            f += len;
            mx = len > mx ? len : mx;
            if (sketch) sk |= __ldg(sketch + k);
        }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
        f += __shfl_xor_sync(0xffffffffu, f, o, 8);
        long long om = __shfl_xor_sync(0xffffffffu, mx, o, 8);
        mx = om > mx ? om : mx;
        sk |= __shfl_xor_sync(0xffffffffu, sk, o, 8);
    }
    if (p < B.nzc && sub == 0) {
        flops[p] = f;
        int64_t cap = f < A.m ? f : A.m;
        int b = bin_of(cap, cfg.warp_max, cfg.block_max);
        bin[p] = (uint8_t)b;
        atomicAdd(&s_cnt[b], 1ull);
        atomicAdd(&s_fl, (unsigned long long)f);
        if (feat) {
            // predictor inputs (see predictor.cu for the definition)
            float d = (float)(be - bs);
            int pc = __popcll(sk);
            float pcf = fminf((float)pc, 63.5f);
            float lc = 64.0f * logf(64.0f / (64.0f - pcf));
            float* x = feat + p * 8;
            x[0] = log1pf(d);
            x[1] = log1pf((float)f);
            x[2] = log1pf((float)mx);
            x[3] = log1pf((float)A.m);
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

void launch_analyze(cudaStream_t st, const DMat& A, const DMat& B, TierCfg cfg, int64_t* flops, uint8_t* bin,
                    unsigned long long* bin_count, unsigned long long* flops_total, const uint64_t* sketch_A,
                    float* feat) {
    if (B.nzc == 0) return;
    int64_t threads = B.nzc * 8;
    int grid = (int)ceil_div64(threads, 256);
    k_analyze<<<grid, 256, 0, st>>>(A, B, cfg, flops, bin, bin_count, flops_total, sketch_A, feat);
    note_launch();
}

// sketch(A(:,k)) = OR over rows i of 2^(bits 31..26 of i * 0x9E3779B1)
__global__ void k_row_sketch(DMat A, uint64_t* __restrict__ sk) {
    int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    int sub = threadIdx.x & 7;
    unsigned long long v = 0;
    if (p < A.nzc) {
        int64_t s = __ldg(A.cp + p), e = __ldg(A.cp + p + 1);
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
    if (A.jc) cudaMemsetAsync(sketch, 0, sizeof(uint64_t) * A.n, st);
    if (A.nzc == 0) return;
    k_row_sketch<<<(int)ceil_div64(A.nzc * 8, 256), 256, 0, st>>>(A, sketch);
    note_launch();
}

// Stable-enough scatter of column ids into per-bin lists (warp-aggregated atomics).
__global__ void k_bin_scatter(int64_t n, const uint8_t* __restrict__ bin, const int64_t* __restrict__ bin_off,
                              unsigned long long* cursor, int32_t* __restrict__ list) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int b = p < n ? bin[p] : -1;
    unsigned mask = __match_any_sync(0xffffffffu, b);
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (b > 0 && lane == leader) base = atomicAdd(cursor + b, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (b > 0) {
        int rank = __popc(mask & ((1u << lane) - 1));
        list[bin_off[b] + base + rank] = (int32_t)p;
    }
}

void launch_bin_scatter(cudaStream_t st, int64_t n, const uint8_t* bin, const int64_t* bin_off,
                        unsigned long long* bin_cursor, int32_t* list) {
    if (n == 0) return;
    k_bin_scatter<<<(int)ceil_div64(n, 256), 256, 0, st>>>(n, bin, bin_off, bin_cursor, list);
    note_launch();
}

__global__ void k_dense_items(const int32_t* __restrict__ dlist, int64_t nd, const int64_t* __restrict__ flops,
                              int G, int part_flops, int2* items, unsigned long long* nitems, int8_t* nparts) {
    int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nd) return;
    int32_t p = dlist[d];
    int64_t f = flops[p];
    int maxp = G < MAX_PARTS ? G : MAX_PARTS;
    int P = (int)std::min<int64_t>(std::max<int64_t>(ceil_div64(f, part_flops), 1), maxp);
    nparts[d] = (int8_t)P;
    unsigned long long base = atomicAdd(nitems, (unsigned long long)P);
    for (int q = 0; q < P; ++q) items[base + q] = make_int2((int)d, q);
}

void launch_dense_items(cudaStream_t st, const int32_t* dense_list, int64_t ndense, const int64_t* flops, int G,
                        int part_flops, int2* items, unsigned long long* nitems, int8_t* nparts) {
    if (ndense == 0) return;
    k_dense_items<<<(int)ceil_div64(ndense, 256), 256, 0, st>>>(dense_list, ndense, flops, G, part_flops, items,
                                                               nitems, nparts);
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

template <class SR, int GS, int TBL, bool NUM, int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_hash(DMat A, DMat B, const int32_t* __restrict__ list, int64_t count,
                                                int64_t* __restrict__ nnz_col, const int64_t* __restrict__ Ccp,
                                                int32_t* __restrict__ Cir, typename SR::T* __restrict__ Cv) {
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

    for (int64_t it = (int64_t)blockIdx.x * NG + g; it < count; it += (int64_t)gridDim.x * NG) {
        const int32_t p = __ldg(list + it);
        const int64_t jout = B.jc ? __ldg(B.jc + p) : p;
        const int64_t bs = __ldg(B.cp + p), be = __ldg(B.cp + p + 1);
        for (int s = lane; s < TBL; s += GS) {
            keys[s] = -1;
            if constexpr (NUM) vals[s] = SR::zero();
        }
        if (lane == 0) *s_cnt = 0;
        G::sync();
        int mycnt = 0;
        for (int64_t b0 = bs; b0 < be; b0 += GS) {
            const int64_t t = b0 + lane;
            int len = 0;
            int64_t a0 = 0;
            T bv = T(0);
            if (t < be) {
                int32_t k = __ldg(B.ir + t);
                int64_t s, e;
                col_range(A, k, s, e);
                a0 = s;
                len = (int)(e - s);
                if constexpr (NUM) bv = load_val<SR>(B, t);
            }
            int total;
            int incl = group_incl_scan<GS>(len, s_scan, total);
            s_incl[lane] = incl;
            s_a0[lane] = a0;
            if constexpr (NUM) s_bv[lane] = bv;
            G::sync();
            for (int e = lane; e < total; e += GS) {
                int lo = 0, hi = GS - 1;
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (s_incl[mid] > e) hi = mid;
                    else lo = mid + 1;
                }
                const int64_t idx = s_a0[lo] + (e - (lo ? s_incl[lo - 1] : 0));
                const int32_t row = __ldg(A.ir + idx);
                uint32_t h = hash_row(row) >> (32 - LOG2);
                while (true) {
                    int32_t cur = vkeys[h];
                    if (cur == row) break;
                    if (cur == -1) {
                        int32_t prev = atomicCAS(&keys[h], -1, row);
                        if (prev == -1) { ++mycnt; break; }
                        if (prev == row) break;
                    }
                    h = (h + 1) & (TBL - 1);
                }
                if constexpr (NUM) SR::atomic_add(&vals[h], SR::mul(load_val<SR>(A, idx), s_bv[lo]));
            }
            G::sync();
        }
        if constexpr (!NUM) {
            int c = warp_sum(mycnt);
            if constexpr (GS == 32) {
                if (lane == 0) nnz_col[jout] = c;
            } else {
                if ((threadIdx.x & 31) == 0) atomicAdd(s_cnt, c);
                __syncthreads();
                if (lane == 0) nnz_col[jout] = *s_cnt;
            }
            G::sync();
        } else {
            const int64_t out0 = __ldg(Ccp + jout);
            const int nnz = (int)(__ldg(Ccp + jout + 1) - out0);
            // in-place compaction toward the front: the i-th occupied slot moves to i <= its slot
            int pos = 0;
            for (int r0 = 0; r0 < TBL; r0 += GS) {
                int s = r0 + lane;
                int32_t k = keys[s];
                Acc v = vals[s];
                int occ = k != -1;
                int total;
                int incl = group_incl_scan<GS>(occ, s_scan, total);
                G::sync();
                if (occ) {
                    keys[pos + incl - 1] = k;
                    vals[pos + incl - 1] = v;
                }
                pos += total;
                G::sync();
            }
            int P = 1;
            while (P < nnz) P <<= 1;
            for (int s = nnz + lane; s < P; s += GS) keys[s] = INT_MAX;
            G::sync();
            bitonic_sort<GS>(keys, vals, P);
            for (int s = lane; s < nnz; s += GS) {
                Cir[out0 + s] = keys[s];
                Cv[out0 + s] = SR::out(vals[s]);
            }
            G::sync();
        }
    }
}

template <class SR, int GS, int TBL, bool NUM, int BLOCK>
static void run_hash(cudaStream_t st, const DMat& A, const DMat& B, const int32_t* list, int64_t count,
                     int64_t* nnz_col, const int64_t* Ccp, int32_t* Cir, typename SR::T* Cv) {
    if (count <= 0) return;
    using L = HashLayout<SR, GS, TBL, NUM>;
    constexpr int NG = BLOCK / GS;
    size_t smem = L::group * NG;
    auto kern = k_hash<SR, GS, TBL, NUM, BLOCK>;
    static bool attr_done = false;   // one attribute call per instantiation
    if (!attr_done) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_done = true;
    }
    int64_t groups = count;
    int64_t want = ceil_div64(groups, NG);
    int grid = (int)std::min<int64_t>(want, 152 * 32);
    kern<<<grid, BLOCK, smem, st>>>(A, B, list, count, nnz_col, Ccp, Cir, Cv);
    note_launch();
}

template <class SR, bool NUM>
static void run_hash_bins(cudaStream_t st, const DMat& A, const DMat& B, const int32_t* list, const int64_t* off,
                          const int64_t* cnt, int64_t* nnz_col, const int64_t* Ccp, int32_t* Cir,
                          typename SR::T* Cv) {
    run_hash<SR, 32, 64, NUM, WARP_BLOCK>(st, A, B, list + off[1], cnt[1], nnz_col, Ccp, Cir, Cv);
    run_hash<SR, 32, 128, NUM, WARP_BLOCK>(st, A, B, list + off[2], cnt[2], nnz_col, Ccp, Cir, Cv);
    run_hash<SR, 32, 256, NUM, WARP_BLOCK>(st, A, B, list + off[3], cnt[3], nnz_col, Ccp, Cir, Cv);
    run_hash<SR, 32, 512, NUM, WARP_BLOCK>(st, A, B, list + off[4], cnt[4], nnz_col, Ccp, Cir, Cv);
    run_hash<SR, 32, 1024, NUM, 128>(st, A, B, list + off[5], cnt[5], nnz_col, Ccp, Cir, Cv);
    run_hash<SR, 256, 2048, NUM, 256>(st, A, B, list + off[6], cnt[6], nnz_col, Ccp, Cir, Cv);
    run_hash<SR, 512, 4096, NUM, 512>(st, A, B, list + off[7], cnt[7], nnz_col, Ccp, Cir, Cv);
    run_hash<SR, 512, 8192, NUM, 512>(st, A, B, list + off[8], cnt[8], nnz_col, Ccp, Cir, Cv);
}

// ------------------------------------------------------------------ dense tier
__device__ __forceinline__ int32_t lower_bound_rows(const int32_t* __restrict__ r, int64_t len, int64_t v) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)__ldg(r + mid) < v) lo = mid + 1;
        else hi = mid;
    }
    return (int32_t)lo;
}

template <class SR, bool NUM>
__global__ void __launch_bounds__(DENSE_BLOCK) k_dense(DMat A, DMat B, const int32_t* __restrict__ dlist,
                                                       int64_t ndense, const int2* __restrict__ items,
                                                       const unsigned long long* __restrict__ nitems_dev, int R, int G,
                                                       const int8_t* __restrict__ nparts, int32_t* __restrict__ cursors,
                                                       int64_t nnzB, int32_t* __restrict__ part_count,
                                                       const int64_t* __restrict__ Ccp, int32_t* __restrict__ Cir,
                                                       typename SR::T* __restrict__ Cv) {
    using Acc = typename SR::Acc;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nw_max = R / 32;
    uint32_t* bitmap = reinterpret_cast<uint32_t*>(smem);
    Acc* vals = reinterpret_cast<Acc*>(smem + (size_t)nw_max * 4);
    int* s_scan = reinterpret_cast<int*>(smem + (size_t)nw_max * 4 + (NUM ? (size_t)R * sizeof(Acc) : 0));
    const int tid = threadIdx.x;
    const int64_t nitems = (int64_t)*nitems_dev;
    if constexpr (NUM) {
        for (int i = tid; i < R; i += DENSE_BLOCK) vals[i] = SR::zero();
    }
    __syncthreads();
    for (int64_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 itm = items[it];
        const int d = itm.x, q = itm.y;
        const int32_t p = __ldg(dlist + d);
        const int P = nparts[d];
        const int64_t jout = B.jc ? __ldg(B.jc + p) : p;
        const int64_t bs = __ldg(B.cp + p), be = __ldg(B.cp + p + 1);
        const int64_t deg = be - bs;
        const int c0 = (int)((int64_t)q * G / P), c1 = (int)((int64_t)(q + 1) * G / P);
        int32_t* cur = cursors + (int64_t)q * nnzB + bs;
        for (int64_t t = tid; t < deg; t += DENSE_BLOCK) {
            int32_t k = __ldg(B.ir + bs + t);
            int64_t s, e;
            col_range(A, k, s, e);
            cur[t] = c0 == 0 ? 0 : lower_bound_rows(A.ir + s, e - s, (int64_t)c0 * R);
        }
        int64_t outpos = 0;
        if constexpr (NUM) {
            outpos = __ldg(Ccp + jout);
            for (int qq = 0; qq < q; ++qq) outpos += part_count[(int64_t)qq * ndense + d];
        }
        int64_t part_total = 0;
        __syncthreads();
        for (int c = c0; c < c1; ++c) {
            const int64_t r0 = (int64_t)c * R;
            const int64_t r1 = std::min<int64_t>(r0 + R, A.m);
            const int nwords = (int)((r1 - r0 + 31) >> 5);
            for (int w = tid; w < nwords; w += DENSE_BLOCK) bitmap[w] = 0u;
            __syncthreads();
            for (int64_t t = tid; t < deg; t += DENSE_BLOCK) {
                const int32_t k = __ldg(B.ir + bs + t);
                int64_t s, e;
                col_range(A, k, s, e);
                int64_t pos = s + cur[t];
                typename SR::T bv = typename SR::T(0);
                if constexpr (NUM) bv = load_val<SR>(B, bs + t);
                while (pos < e) {
                    const int32_t r = __ldg(A.ir + pos);
                    if (r >= r1) break;
                    if (r < r0) { ++pos; continue; }   // only on unsorted (malformed) columns
                    const int lr = (int)(r - r0);
                    atomicOr(&bitmap[lr >> 5], 1u << (lr & 31));
                    if constexpr (NUM) SR::atomic_add(&vals[lr], SR::mul(load_val<SR>(A, pos), bv));
                    ++pos;
                }
                cur[t] = (int32_t)(pos - s);
            }
            __syncthreads();
            const int wpt = (nwords + DENSE_BLOCK - 1) / DENSE_BLOCK;
            const int w0 = tid * wpt, w1 = std::min(w0 + wpt, nwords);
            int cnt = 0;
            for (int w = w0; w < w1; ++w) cnt += __popc(bitmap[w]);
            int total;
            int incl = group_incl_scan<DENSE_BLOCK>(cnt, s_scan, total);
            if constexpr (NUM) {
                int64_t o = outpos + incl - cnt;
                for (int w = w0; w < w1; ++w) {
                    uint32_t bits = bitmap[w];
                    while (bits) {
                        int b = __ffs(bits) - 1;
                        bits &= bits - 1;
                        int lr = w * 32 + b;
                        Cir[o] = (int32_t)(r0 + lr);
                        Cv[o] = SR::out(vals[lr]);
                        vals[lr] = SR::zero();
                        ++o;
                    }
                }
            }
            outpos += total;
            part_total += total;
            __syncthreads();
        }
        if constexpr (!NUM) {
            if (tid == 0) part_count[(int64_t)q * ndense + d] = (int32_t)part_total;
        }
    }
}

template <class SR, bool NUM>
static void run_dense(cudaStream_t st, const DMat& A, const DMat& B, int R, const int32_t* dlist, int64_t ndense,
                      const int2* items, const unsigned long long* nitems, int64_t nitems_host, const int8_t* nparts,
                      int32_t* cursors, int32_t* part_count, const int64_t* Ccp, int32_t* Cir,
                      typename SR::T* Cv) {
    if (ndense <= 0 || A.m == 0) return;
    const int G = (int)ceil_div64(A.m, R);
    size_t smem = (size_t)(R / 32) * 4 + (NUM ? (size_t)R * sizeof(typename SR::Acc) : 0) + 34 * 4;
    auto kern = k_dense<SR, NUM>;
    static size_t attr_done = 0;
    if (attr_done < smem) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_done = smem;
    }
    int64_t want = nitems_host > 0 ? nitems_host : ndense * MAX_PARTS;
    int grid = (int)std::min<int64_t>(want, 152 * 8);
    kern<<<grid, DENSE_BLOCK, smem, st>>>(A, B, dlist, ndense, items, nitems, R, G, nparts, cursors, B.nnz,
                                          part_count, Ccp, Cir, Cv);
    note_launch();
}

template <class SR>
void launch_symbolic(cudaStream_t st, const DMat& A, const DMat& B, TierCfg cfg, const int32_t* list,
                     const int64_t* bin_off, const int64_t* bin_cnt, const int2* dense_items,
                     const unsigned long long* nitems, int64_t nitems_host, const int8_t* nparts, int32_t* cursors,
                     int32_t* part_count, int64_t* nnz_col, int which) {
    if (which & 1) run_hash_bins<SR, false>(st, A, B, list, bin_off, bin_cnt, nnz_col, nullptr, nullptr, nullptr);
    if (which & 2) run_dense<SR, false>(st, A, B, cfg.dense_rows, list + bin_off[BIN_DENSE], bin_cnt[BIN_DENSE], dense_items, nitems,
                         nitems_host, nparts, cursors, part_count, nullptr, nullptr, nullptr);
}

template <class SR>
void launch_numeric(cudaStream_t st, const DMat& A, const DMat& B, TierCfg cfg, const int32_t* list,
                    const int64_t* bin_off, const int64_t* bin_cnt, const int2* dense_items,
                    const unsigned long long* nitems, int64_t nitems_host, int32_t* cursors,
                    const int32_t* part_count, const int8_t* nparts, const int64_t* Ccp, int32_t* Cir,
                    typename SR::T* Cv, int which) {
    if (which & 1) run_hash_bins<SR, true>(st, A, B, list, bin_off, bin_cnt, nullptr, Ccp, Cir, Cv);
    if (which & 2) run_dense<SR, true>(st, A, B, cfg.dense_rows, list + bin_off[BIN_DENSE], bin_cnt[BIN_DENSE], dense_items, nitems,
                        nitems_host, nparts, cursors, const_cast<int32_t*>(part_count), Ccp, Cir, Cv);
}

#define SG_INST(SR)                                                                                              \
    template void launch_symbolic<SR>(cudaStream_t, const DMat&, const DMat&, TierCfg, const int32_t*,           \
                                      const int64_t*, const int64_t*, const int2*, const unsigned long long*,    \
                                      int64_t, const int8_t*, int32_t*, int32_t*, int64_t*, int);                                    \
    template void launch_numeric<SR>(cudaStream_t, const DMat&, const DMat&, TierCfg, const int32_t*,            \
                                     const int64_t*, const int64_t*, const int2*, const unsigned long long*,     \
                                     int64_t, int32_t*, const int32_t*, const int8_t*, const int64_t*, int32_t*, \
                                     typename SR::T*, int);
SG_INST(PT64)
SG_INST(MP32)
SG_INST(BOOL8)
SG_INST(PTI64)
#undef SG_INST

// ------------------------------------------------------------------ part sums, fills, scan
__global__ void k_sum_parts(const int32_t* __restrict__ dlist, int64_t nd, const int8_t* __restrict__ nparts,
                            const int32_t* __restrict__ pc, int64_t* __restrict__ nnz_col, const int32_t* __restrict__ jc) {
    int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= nd) return;
    int P = nparts[d];
    int64_t s = 0;
    for (int q = 0; q < P; ++q) s += pc[(int64_t)q * nd + d];
    int32_t p = dlist[d];
    nnz_col[jc ? jc[p] : p] = s;
}

void launch_sum_parts(cudaStream_t st, const int32_t* dense_list, int64_t ndense, const int8_t* nparts,
                      const int32_t* part_count, int64_t* nnz_col, const int32_t* jc) {
    if (ndense == 0) return;
    k_sum_parts<<<(int)ceil_div64(ndense, 256), 256, 0, st>>>(dense_list, ndense, nparts, part_count, nnz_col, jc);
    note_launch();
}

__global__ void k_fill_i64(int64_t* p, int64_t n, int64_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

void launch_fill_i64(cudaStream_t st, int64_t* p, int64_t n, int64_t v) {
    if (n <= 0) return;
    int grid = (int)std::min<int64_t>(ceil_div64(n, 256), 152 * 16);
    k_fill_i64<<<grid, 256, 0, st>>>(p, n, v);
    note_launch();
}

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

__global__ void k_tier_stats(const uint8_t* __restrict__ bin, const int64_t* __restrict__ flops,
                             const int64_t* __restrict__ nnz_col, const int32_t* __restrict__ jc,
                             const int64_t* __restrict__ bcp, int64_t nzc, unsigned long long* out) {
    __shared__ unsigned long long s[16];
    if (threadIdx.x < 16) s[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nzc; p += (int64_t)gridDim.x * blockDim.x) {
        int b = bin[p];
        int t = b == 0 ? 0 : (b <= NWARP ? 1 : (b < BIN_DENSE ? 2 : 3));
        atomicAdd(&s[t], 1ull);
        atomicAdd(&s[4 + t], (unsigned long long)flops[p]);
        atomicAdd(&s[8 + t], (unsigned long long)nnz_col[jc ? jc[p] : p]);
        atomicAdd(&s[12 + t], (unsigned long long)(bcp[p + 1] - bcp[p]));
    }
    __syncthreads();
    if (threadIdx.x < 16 && s[threadIdx.x]) atomicAdd(out + threadIdx.x, s[threadIdx.x]);
}

void launch_tier_stats(cudaStream_t st, const uint8_t* bin, const int64_t* flops, const int64_t* nnz_col,
                       const int32_t* jc, const int64_t* bcp, int64_t nzc, unsigned long long* out) {
    if (nzc <= 0) return;
    int grid = (int)std::min<int64_t>(ceil_div64(nzc, 256), 152 * 4);
    k_tier_stats<<<grid, 256, 0, st>>>(bin, flops, nnz_col, jc, bcp, nzc, out);
    note_launch();
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
    note_launch();
    k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(sums, nb);
    note_launch();
    k_scan_apply<<<(int)nb, SCAN_BLOCK, 0, st>>>(in, n, sums, out);
    note_launch();
}

}  // namespace sg
