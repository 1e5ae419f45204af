// Format conversions: transpose (Section 2.4 transposes B once as a
// preprocessing step), CSC -> DCSC with the AUX column index (Section 2.3),
// and device-side validation of the CSC invariants.
#include <algorithm>

#include "internal.cuh"

using namespace sg;

namespace {

constexpr int RS_BLOCK = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_BLOCK * RS_ROUNDS;
constexpr int RS_WARPS = RS_BLOCK / 32;

// ---------------------------------------------------------------- stable LSD radix sort
// (uint32 key, uint32 payload) pairs, 8-bit digits.  Tile order inside a CTA is
// element e = round * 256 + tid, ranks are assigned in that order, so each pass is
// stable and the passes compose into a stable sort.
__global__ void __launch_bounds__(RS_BLOCK) k_rs_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                      int64_t ntiles, int64_t* __restrict__ hist) {
    __shared__ int cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t e = t0 + r * RS_BLOCK + threadIdx.x;
        if (e < n) atomicAdd(&cnt[(keys[e] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(RS_BLOCK) k_rs_scatter(const uint32_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin, int64_t n, int shift,
                                                         int64_t ntiles, const int64_t* __restrict__ off,
                                                         uint32_t* __restrict__ kout, uint32_t* __restrict__ vout) {
    __shared__ int run[256];
    __shared__ int wcnt[RS_WARPS][256];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    run[tid] = 0;
    const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const int64_t e = t0 + r * RS_BLOCK + tid;
        const bool valid = e < n;
        uint32_t key = valid ? kin[e] : 0u;
        uint32_t val = valid ? vin[e] : 0u;
        int d = valid ? (int)((key >> shift) & 255u) : 256;
        unsigned mask = __match_any_sync(0xffffffffu, d);
        int rank = __popc(mask & ((1u << lane) - 1u));
        int leader = __ffs(mask) - 1;
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ++ww) wcnt[ww][tid] = 0;
        __syncthreads();
        if (valid && lane == leader) wcnt[w][d] = __popc(mask);
        __syncthreads();
        {
            int acc = run[tid];
#pragma unroll
            for (int ww = 0; ww < RS_WARPS; ++ww) {
                int c = wcnt[ww][tid];
                wcnt[ww][tid] = acc;
                acc += c;
            }
            run[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = off[(int64_t)d * ntiles + blockIdx.x] + wcnt[w][d] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
    }
}

__global__ void k_iota_u32(uint32_t* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (uint32_t)i;
}

__global__ void k_expand_cols(const int64_t* __restrict__ cp, int64_t n, int32_t* __restrict__ col) {
    int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    int sub = threadIdx.x & 7;
    if (j >= n) return;
    for (int64_t t = cp[j] + sub; t < cp[j + 1]; t += 8) col[t] = (int32_t)j;
}

__global__ void k_row_hist(const int32_t* __restrict__ ir, int64_t nnz, int64_t m, int64_t* __restrict__ cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x)
        if (ir[i] >= 0 && ir[i] < m) atomicAdd(reinterpret_cast<unsigned long long*>(cnt + ir[i]), 1ull);
}

template <int W>
struct Word;
template <>
struct Word<1> { using T = uint8_t; };
template <>
struct Word<4> { using T = uint32_t; };
template <>
struct Word<8> { using T = uint64_t; };

template <int W>
__global__ void k_gather(const uint32_t* __restrict__ perm, const int32_t* __restrict__ colid,
                         const void* __restrict__ vin, int64_t nnz, int32_t* __restrict__ ir_out,
                         void* __restrict__ vout) {
    using T = typename Word<W>::T;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t s = perm[i];
        ir_out[i] = colid[s];
        if (vin) reinterpret_cast<T*>(vout)[i] = reinterpret_cast<const T*>(vin)[s];
    }
}

int grid_for(int64_t n, int block = 256) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div64(n, block), sm_count() * 32)); }

// ---------------------------------------------------------------- DCSC
__global__ void k_nonempty(const int64_t* __restrict__ cp, int64_t n, int64_t* __restrict__ flag) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        flag[j] = cp[j + 1] > cp[j] ? 1 : 0;
}

__global__ void k_dcsc_scatter(const int64_t* __restrict__ cp, int64_t n, const int64_t* __restrict__ pos,
                               int32_t* __restrict__ jc, int64_t* __restrict__ dcp) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        if (cp[j + 1] > cp[j]) {
            jc[pos[j]] = (int32_t)j;
            dcp[pos[j]] = cp[j];
        }
        if (j == n - 1) dcp[pos[n]] = cp[n];
    }
}

// AUX[t] = first JC position whose column id >= t * chunk; AUX[naux] = nzc
__global__ void k_aux(const int32_t* __restrict__ jc, int64_t nzc, int64_t chunk, int64_t naux,
                      int32_t* __restrict__ aux) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= naux; t += (int64_t)gridDim.x * blockDim.x) {
        if (t == naux) {
            aux[t] = (int32_t)nzc;
            continue;
        }
        int64_t v = t * chunk, lo = 0, hi = nzc;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if ((int64_t)jc[mid] < v) lo = mid + 1;
            else hi = mid;
        }
        aux[t] = (int32_t)lo;
    }
}

// ---------------------------------------------------------------- validation
__global__ void k_validate(const int64_t* __restrict__ cp, const int32_t* __restrict__ ir, int64_t m, int64_t n,
                           int64_t nnz, int* __restrict__ bad) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = cp[j], e = cp[j + 1];
        if (j == 0 && s != 0) { atomicMax(bad, 1); continue; }
        if (j == n - 1 && e != nnz) { atomicMax(bad, 2); continue; }
        if (e < s || s < 0 || e > nnz) { atomicMax(bad, 3); continue; }
        int32_t prev = -1;
        for (int64_t t = s; t < e; ++t) {
            int32_t r = ir[t];
            if (r < 0 || r >= m) { atomicMax(bad, 4); break; }
            if (r <= prev) { atomicMax(bad, 5); break; }
            prev = r;
        }
    }
}

// Format check of several stored CSC arrays at once: one warp per column of the
// concatenated column space (handle h owns columns [cbase[h], cbase[h+1])); the
// first lane checks the column's pointers, all lanes its rows.  bad[h] gets the
// largest violation code seen.
struct VDesc {
    const int64_t* cp;
    const int32_t* ir;
    int64_t m, n, nnz;
};
__global__ void k_validate_many(const VDesc* __restrict__ d, const int64_t* __restrict__ cbase, int nh,
                                int* __restrict__ bad) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = cbase[nh];
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < total; c += nwarps) {
        int lo = 0, hi = nh - 1;   // the handle h with cbase[h] <= c < cbase[h+1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cbase[mid] <= c) lo = mid;
            else hi = mid - 1;
        }
        const VDesc D = d[lo];
        const int64_t j = c - cbase[lo];
        const int64_t s = D.cp[j], e = D.cp[j + 1];
        int code = 0;
        if (j == 0 && s != 0) code = 1;
        else if (j == D.n - 1 && e != D.nnz) code = 2;
        else if (e < s || s < 0 || e > D.nnz) code = 3;
        if (code == 0) {
            for (int64_t t = s + lane; t < e; t += 32) {
                const int32_t r = D.ir[t];
                if (r < 0 || r >= D.m) code = code > 4 ? code : 4;
                else if (t > s && D.ir[t - 1] >= r) code = 5;
            }
        }
        if (code) atomicMax(bad + lo, code);
    }
}

}  // namespace

spgemm_status_t check_handles(spgemm_ctx* ctx, const std::vector<spgemm_mat*>& mats) {
    std::vector<spgemm_mat*> todo;
    for (spgemm_mat* M : mats)
        if (M && !M->checked && M->fmt != SPGEMM_FMT_DCSC && std::find(todo.begin(), todo.end(), M) == todo.end())
            todo.push_back(M);
    if (todo.empty()) return SPGEMM_OK;
    const int nh = (int)todo.size();
    std::vector<VDesc> hd(nh);
    std::vector<int64_t> hb(nh + 1, 0);
    for (int h = 0; h < nh; ++h) {
        spgemm_mat* M = todo[h];
        // stored arrays: CSC of (rows = stored m) x (cols = stored n)
        const int64_t sm = M->fmt == SPGEMM_FMT_CSR ? M->n : M->m;
        const int64_t sn = M->fmt == SPGEMM_FMT_CSR ? M->m : M->n;
        hd[h] = VDesc{M->cp, M->ir, sm, sn, M->nnz};
        hb[h + 1] = hb[h] + sn;
    }
    const size_t bytes = sizeof(VDesc) * nh + 8 * (nh + 1) + 4 * nh;
    auto buf = ctx_buf(ctx, bytes);
    if (!buf) return set_err(ctx, SPGEMM_ERR_OOM, "input check");
    VDesc* dd = (VDesc*)buf->p;
    int64_t* db = (int64_t*)(dd + nh);
    int* dbad = (int*)(db + nh + 1);
    cudaStream_t st = ctx->stream;
    SG_CUDA(ctx, cudaMemcpyAsync(dd, hd.data(), sizeof(VDesc) * nh, cudaMemcpyHostToDevice, st));
    SG_CUDA(ctx, cudaMemcpyAsync(db, hb.data(), 8 * (nh + 1), cudaMemcpyHostToDevice, st));
    SG_CUDA(ctx, cudaMemsetAsync(dbad, 0, 4 * nh, st));
    std::vector<int> hbad(nh, 0);
    if (hb[nh] > 0) {
        k_validate_many<<<grid_for(hb[nh] * 32), 256, 0, st>>>(dd, db, nh, dbad);
        note_launch();
    }
    SG_TRY(read_back(ctx, hbad.data(), dbad, 4 * nh));
    // a matrix without columns: its (single) column pointer must be 0 and nnz 0
    std::vector<int64_t> c0(nh, 0);
    for (int h = 0; h < nh; ++h)
        if (hb[h + 1] == hb[h]) SG_TRY(read_back(ctx, &c0[h], todo[h]->cp, 8));
    SG_TRY(sync_ctx(ctx));
    static const char* why[] = {"", "colptr[0] != 0", "colptr[n] != nnz", "colptr not monotone",
                                "row index out of range", "rows not strictly ascending in a column"};
    for (int h = 0; h < nh; ++h) {
        int code = hbad[h];
        if (hb[h + 1] == hb[h] && (c0[h] != 0 || todo[h]->nnz != 0)) code = 1;
        if (code)
            return set_err(ctx, SPGEMM_ERR_BAD_FORMAT, "operand %d of this call (%lld x %lld): %s", h,
                           (long long)todo[h]->m, (long long)todo[h]->n, why[code < 6 ? code : 0]);
    }
    for (spgemm_mat* M : todo) M->checked = true;
    return SPGEMM_OK;
}

// Stable sort of (key, payload) pairs by the low `bits` bits of key, LSD with
// 8-bit digits.  Buffers (k0, v0) hold the input; the result ends in (k0, v0)
// or (k1, v1): *in_second tells which.  tmp needs radix_tmp_bytes(n).
size_t radix_tmp_bytes(int64_t n) {
    const int64_t ntiles = std::max<int64_t>(1, ceil_div64(n, RS_TILE));
    return 8 * (256 * ntiles + 1) * 2 + scan_tmp_bytes(256 * ntiles) + 256;
}

void radix_sort_pairs(cudaStream_t st, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int64_t n, int bits,
                      void* tmp, bool* in_second) {
    *in_second = false;
    if (n <= 0 || bits <= 0) return;
    const int64_t ntiles = std::max<int64_t>(1, ceil_div64(n, RS_TILE));
    int64_t* hist = (int64_t*)tmp;
    int64_t* off = hist + (256 * ntiles + 1);
    void* stmp = off + (256 * ntiles + 1);
    for (int shift = 0; shift < bits; shift += 8) {
        k_rs_hist<<<(int)ntiles, RS_BLOCK, 0, st>>>(k0, n, shift, ntiles, hist);
        note_launch();
        launch_exclusive_scan(st, hist, 256 * ntiles, off, stmp);
        k_rs_scatter<<<(int)ntiles, RS_BLOCK, 0, st>>>(k0, v0, n, shift, ntiles, off, k1, v1);
        note_launch();
        std::swap(k0, k1);
        std::swap(v0, v1);
        *in_second = !*in_second;
    }
}

// CSC (m x n) -> CSC of the transpose (n x m), rows sorted.  `out` is filled in place.
spgemm_status_t transpose_csc(spgemm_ctx* ctx, int64_t m, int64_t n, int64_t nnz, const int64_t* cp,
                              const int32_t* ir, const void* num, size_t w, spgemm_mat_t out) {
    cudaStream_t st = ctx->stream;
    if (nnz > (int64_t)UINT32_MAX) return set_err(ctx, SPGEMM_ERR_INDEX_OVERFLOW, "transpose: nnz beyond 2^32");
    const int64_t ntiles = std::max<int64_t>(1, ceil_div64(nnz, RS_TILE));
    auto cpb = ctx_buf(ctx, 8 * (m + 1));
    auto irb = ctx_buf(ctx, 4 * std::max<int64_t>(nnz, 1));
    auto vb = ctx_buf(ctx, w * std::max<int64_t>(nnz, 1));
    size_t tmp_bytes = 4 * 4 * std::max<int64_t>(nnz, 1) + 4 * std::max<int64_t>(nnz, 1) +
                       8 * (256 * ntiles + 1) * 2 + scan_tmp_bytes(std::max<int64_t>(256 * ntiles, m)) + 8 * (m + 1) +
                       1024;
    auto tmp = ctx_buf(ctx, tmp_bytes);
    if (!cpb || !irb || !vb || !tmp) return set_err(ctx, SPGEMM_ERR_OOM, "transpose buffers");
    char* t = (char*)tmp->p;
    const int64_t nz1 = std::max<int64_t>(nnz, 1);
    uint32_t* k0 = (uint32_t*)t; t += 4 * nz1;
    uint32_t* k1 = (uint32_t*)t; t += 4 * nz1;
    uint32_t* v0 = (uint32_t*)t; t += 4 * nz1;
    uint32_t* v1 = (uint32_t*)t; t += 4 * nz1;
    int32_t* colid = (int32_t*)t; t += 4 * nz1;
    t = (char*)(((uintptr_t)t + 255) / 256 * 256);
    int64_t* hist = (int64_t*)t; t += 8 * (256 * ntiles + 1);
    int64_t* off = (int64_t*)t; t += 8 * (256 * ntiles + 1);
    int64_t* rowcnt = (int64_t*)t; t += 8 * (m + 1);
    void* stmp = t;
    int64_t* tcp = (int64_t*)cpb->p;
    if (nnz > 0) {
        SG_CUDA(ctx, cudaMemcpyAsync(k0, ir, 4 * nnz, cudaMemcpyDeviceToDevice, st));
        k_iota_u32<<<grid_for(nnz), 256, 0, st>>>(v0, nnz);
        note_launch();
        k_expand_cols<<<(int)ceil_div64(n * 8, 256) + 1, 256, 0, st>>>(cp, n, colid);
        note_launch();
        int bits = 0;
        while (bits < 32 && (int64_t(1) << bits) < m) ++bits;
        for (int shift = 0; shift < bits; shift += 8) {
            k_rs_hist<<<(int)ntiles, RS_BLOCK, 0, st>>>(k0, nnz, shift, ntiles, hist);
            note_launch();
            launch_exclusive_scan(st, hist, 256 * ntiles, off, stmp);
            k_rs_scatter<<<(int)ntiles, RS_BLOCK, 0, st>>>(k0, v0, nnz, shift, ntiles, off, k1, v1);
            note_launch();
            std::swap(k0, k1);
            std::swap(v0, v1);
        }
        SG_CUDA(ctx, cudaMemsetAsync(rowcnt, 0, 8 * m, st));
        k_row_hist<<<grid_for(nnz), 256, 0, st>>>(ir, nnz, m, rowcnt);
        note_launch();
        launch_exclusive_scan(st, rowcnt, m, tcp, stmp);
        note_launch();
        switch (w) {
        case 1: k_gather<1><<<grid_for(nnz), 256, 0, st>>>(v0, colid, num, nnz, (int32_t*)irb->p, vb->p); break;
        case 4: k_gather<4><<<grid_for(nnz), 256, 0, st>>>(v0, colid, num, nnz, (int32_t*)irb->p, vb->p); break;
        default: k_gather<8><<<grid_for(nnz), 256, 0, st>>>(v0, colid, num, nnz, (int32_t*)irb->p, vb->p); break;
        }
    } else {
        SG_CUDA(ctx, cudaMemsetAsync(tcp, 0, 8 * (m + 1), st));
    }
    SG_CUDA(ctx, cudaGetLastError());
    out->ctx = ctx;
    out->fmt = SPGEMM_FMT_CSC;
    out->m = n;
    out->n = m;
    out->nnz = nnz;
    out->nzc = m;
    out->cp = tcp;
    out->ir = (const int32_t*)irb->p;
    out->num = num ? vb->p : nullptr;
    out->owned = {cpb, irb, vb, tmp};
    // the temporaries are released with the handle's first owner release; drop them now
    out->owned.pop_back();
    return SPGEMM_OK;
}

spgemm_status_t make_dcsc(spgemm_ctx* ctx, const spgemm_mat* M, bool with_aux, spgemm_mat* out) {
    cudaStream_t st = ctx->stream;
    const int64_t n = M->n;
    auto tmp = ctx_buf(ctx, 8 * (n + 1) * 2 + scan_tmp_bytes(n));
    if (!tmp) return set_err(ctx, SPGEMM_ERR_OOM, "dcsc temporaries");
    int64_t* flag = (int64_t*)tmp->p;
    int64_t* pos = flag + (n + 1);
    void* stmp = pos + (n + 1);
    int64_t nzc = 0;
    if (n > 0) {
        k_nonempty<<<grid_for(n), 256, 0, st>>>(M->cp, n, flag);
        note_launch();
        launch_exclusive_scan(st, flag, n, pos, stmp);
        SG_TRY(read_back(ctx, &nzc, pos + n, 8));
        SG_TRY(sync_ctx(ctx));
    }
    const int64_t chunk = n == 0 ? 1 : (nzc > 0 ? ceil_div64(n, nzc) : n);
    const int64_t naux = n == 0 ? 0 : ceil_div64(n, chunk);
    auto jcb = ctx_buf(ctx, 4 * std::max<int64_t>(nzc, 1));
    auto cpb = ctx_buf(ctx, 8 * (nzc + 1));
    std::shared_ptr<DevBuf> auxb;
    if (with_aux) auxb = ctx_buf(ctx, 4 * (naux + 1));
    if (!jcb || !cpb || (with_aux && !auxb)) return set_err(ctx, SPGEMM_ERR_OOM, "dcsc arrays");
    if (n > 0) {
        k_dcsc_scatter<<<grid_for(n), 256, 0, st>>>(M->cp, n, pos, (int32_t*)jcb->p, (int64_t*)cpb->p);
        note_launch();
    } else {
        SG_CUDA(ctx, cudaMemsetAsync(cpb->p, 0, 8, st));
    }
    if (with_aux) {
        k_aux<<<grid_for(naux + 1), 256, 0, st>>>((int32_t*)jcb->p, nzc, chunk, naux, (int32_t*)auxb->p);
        note_launch();
    }
    SG_CUDA(ctx, cudaGetLastError());
    out->ctx = ctx;
    out->fmt = SPGEMM_FMT_DCSC;
    out->sr = M->sr;
    out->m = M->m;
    out->n = n;
    out->nnz = M->nnz;
    out->nzc = nzc;
    out->cp = (const int64_t*)cpb->p;
    out->jc = (const int32_t*)jcb->p;
    out->aux = with_aux ? (const int32_t*)auxb->p : nullptr;
    out->naux = with_aux ? naux : 0;
    out->chunk = chunk;
    out->ir = M->ir;
    out->num = M->num;
    out->owned = M->owned;   // share the source's arrays if it owns them
    out->owned.push_back(jcb);
    out->owned.push_back(cpb);
    if (auxb) out->owned.push_back(auxb);
    return SPGEMM_OK;
}

// ------------------------------------------------------------------ permutation
// B = P A Q^T, B(p[i], q[j]) = A(i, j): the relabelling behind the random symmetric
// permutation of Section 5.3.3 (C' = (PAP^T)(PBP^T) = PCP^T) used to balance the 2D grid.

// counts[v]++ for every permutation entry; entries outside [0, n) raise the flag
__global__ void k_perm_count(const int32_t* __restrict__ perm, int64_t n, int32_t* __restrict__ cnt, int* bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = perm[i];
        if (v < 0 || v >= n) atomicExch(bad, 1);
        else atomicAdd(cnt + v, 1);
    }
}

// a permutation hits every value exactly once
__global__ void k_perm_check(const int32_t* __restrict__ cnt, int64_t n, int* bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (cnt[i] != 1) atomicExch(bad, 1);
}

// first sort key: the new row p[ir[t]] of every entry, and the entry index
__global__ void k_perm_rows(const int32_t* __restrict__ ir, const int32_t* __restrict__ rowp, int64_t nnz,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ idx) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = ir[t];
        key[t] = (uint32_t)(rowp ? rowp[r] : r);
        idx[t] = (uint32_t)t;
    }
}

// second sort key: the new column q[col(t)] of the entries in their row-sorted order
__global__ void k_perm_cols(const uint32_t* __restrict__ idx, const int32_t* __restrict__ colid,
                            const int32_t* __restrict__ colp, int64_t nnz, uint32_t* __restrict__ key,
                            int64_t* __restrict__ colcnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = colid[idx[i]];
        const uint32_t nc = (uint32_t)(colp ? colp[c] : c);
        key[i] = nc;
        atomicAdd(reinterpret_cast<unsigned long long*>(colcnt + nc), 1ull);
    }
}

template <int W>
__global__ void k_perm_gather(const uint32_t* __restrict__ idx, const int32_t* __restrict__ ir,
                              const int32_t* __restrict__ rowp, const void* __restrict__ vin, int64_t nnz,
                              int32_t* __restrict__ ir_out, void* __restrict__ vout) {
    using T = typename Word<W>::T;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = idx[i];
        const int32_t r = ir[t];
        ir_out[i] = rowp ? rowp[r] : r;
        if (vin) reinterpret_cast<T*>(vout)[i] = reinterpret_cast<const T*>(vin)[t];
    }
}

static int bits_for(int64_t n) {
    int b = 0;
    while (b < 32 && (int64_t(1) << b) < n) ++b;
    return b;
}

// Checks that perm (n entries) is a permutation of 0..n-1 (synchronises the stream).
static spgemm_status_t check_perm(spgemm_ctx* ctx, const int32_t* perm, int64_t n, const char* what) {
    if (!perm || n == 0) return SPGEMM_OK;
    cudaStream_t st = ctx->stream;
    auto b = ctx_buf(ctx, 4 * n + 16);
    if (!b) return set_err(ctx, SPGEMM_ERR_OOM, "permutation check");
    int32_t* cnt = (int32_t*)b->p;
    int* bad = (int*)(cnt + n);
    SG_CUDA(ctx, cudaMemsetAsync(b->p, 0, 4 * n + 16, st));
    k_perm_count<<<grid_for(n), 256, 0, st>>>(perm, n, cnt, bad);
    k_perm_check<<<grid_for(n), 256, 0, st>>>(cnt, n, bad);
    note_launch(2);
    int h = 0;
    SG_TRY(read_back(ctx, &h, bad, sizeof(int)));
    SG_TRY(sync_ctx(ctx));
    if (h) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "%s is not a permutation of 0..%lld", what, (long long)(n - 1));
    return SPGEMM_OK;
}

static spgemm_status_t permute_csc(spgemm_ctx* ctx, int64_t m, int64_t n, int64_t nnz, const int64_t* cp,
                                   const int32_t* ir, const void* num, size_t w, const int32_t* rowp,
                                   const int32_t* colp, spgemm_mat* out) {
    cudaStream_t st = ctx->stream;
    if (nnz > (int64_t)UINT32_MAX) return set_err(ctx, SPGEMM_ERR_INDEX_OVERFLOW, "permute: nnz beyond 2^32");
    const int64_t nz1 = std::max<int64_t>(nnz, 1);
    auto cpb = ctx_buf(ctx, 8 * (n + 1));
    auto irb = ctx_buf(ctx, 4 * nz1);
    auto vb = ctx_buf(ctx, w * nz1);
    const size_t rs = radix_tmp_bytes(nnz);
    auto tmp = ctx_buf(ctx, 5 * 4 * nz1 + 8 * (n + 1) + rs + scan_tmp_bytes(std::max<int64_t>(n, 1)) + 1024);
    if (!cpb || !irb || !vb || !tmp) return set_err(ctx, SPGEMM_ERR_OOM, "permute buffers");
    char* t = (char*)tmp->p;
    uint32_t* k0 = (uint32_t*)t; t += 4 * nz1;
    uint32_t* k1 = (uint32_t*)t; t += 4 * nz1;
    uint32_t* v0 = (uint32_t*)t; t += 4 * nz1;
    uint32_t* v1 = (uint32_t*)t; t += 4 * nz1;
    int32_t* colid = (int32_t*)t; t += 4 * nz1;
    t = (char*)(((uintptr_t)t + 255) / 256 * 256);
    int64_t* colcnt = (int64_t*)t; t += 8 * (n + 1);
    t = (char*)(((uintptr_t)t + 255) / 256 * 256);
    void* rtmp = t; t += rs;
    t = (char*)(((uintptr_t)t + 255) / 256 * 256);
    void* stmp = t;
    int64_t* ocp = (int64_t*)cpb->p;
    SG_CUDA(ctx, cudaMemsetAsync(colcnt, 0, 8 * (n + 1), st));
    if (nnz > 0) {
        // LSD order: by new row, then stably by new column
        k_perm_rows<<<grid_for(nnz), 256, 0, st>>>(ir, rowp, nnz, k0, v0);
        k_expand_cols<<<(int)ceil_div64(n * 8, 256) + 1, 256, 0, st>>>(cp, n, colid);
        note_launch(2);
        bool second = false;
        radix_sort_pairs(st, k0, v0, k1, v1, nnz, bits_for(m), rtmp, &second);
        uint32_t* vr = second ? v1 : v0;   // entry indices in new-row order
        uint32_t* kA = second ? k0 : k1;   // free key buffer
        uint32_t* kB = second ? k1 : k0;   // the row keys, no longer needed
        uint32_t* vB = second ? v0 : v1;   // free value buffer
        k_perm_cols<<<grid_for(nnz), 256, 0, st>>>(vr, colid, colp, nnz, kA, colcnt);
        note_launch();
        bool second2 = false;
        radix_sort_pairs(st, kA, vr, kB, vB, nnz, bits_for(n), rtmp, &second2);
        const uint32_t* fin = second2 ? vB : vr;
        switch (w) {
        case 1: k_perm_gather<1><<<grid_for(nnz), 256, 0, st>>>(fin, ir, rowp, num, nnz, (int32_t*)irb->p, vb->p); break;
        case 4: k_perm_gather<4><<<grid_for(nnz), 256, 0, st>>>(fin, ir, rowp, num, nnz, (int32_t*)irb->p, vb->p); break;
        default: k_perm_gather<8><<<grid_for(nnz), 256, 0, st>>>(fin, ir, rowp, num, nnz, (int32_t*)irb->p, vb->p); break;
        }
        note_launch();
    }
    launch_exclusive_scan(st, colcnt, n, ocp, stmp);
    SG_CUDA(ctx, cudaGetLastError());
    out->ctx = ctx;
    out->fmt = SPGEMM_FMT_CSC;
    out->m = m;
    out->n = n;
    out->nnz = nnz;
    out->nzc = n;
    out->cp = ocp;
    out->ir = (const int32_t*)irb->p;
    out->num = num ? vb->p : nullptr;
    out->owned = {cpb, irb, vb};
    SG_TRY(sync_ctx(ctx));   // the temporaries are released when this call returns
    return SPGEMM_OK;
}

extern "C" {

spgemm_status_t spgemm_mat_permute(spgemm_ctx_t ctx, spgemm_mat_t a, const int32_t* row_perm,
                                   const int32_t* col_perm, spgemm_mat_t* out) {
    if (!ctx || !a || !out) return SPGEMM_ERR_INVALID_ARG;
    if (a->fmt == SPGEMM_FMT_DCSC) return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "permute of a DCSC handle");
    SG_TRY(check_perm(ctx, row_perm, a->m, "row_perm"));
    SG_TRY(check_perm(ctx, col_perm, a->n, "col_perm"));
    SG_TRY(check_handles(ctx, {a}));
    spgemm_mat_t conv = nullptr;
    DMat d;
    SG_TRY(to_csc_operand(ctx, a, &conv, &d));
    std::unique_ptr<spgemm_mat> hold(conv);
    auto* P = new spgemm_mat();
    spgemm_status_t s = permute_csc(ctx, d.m, d.n, d.nnz, d.cp, d.ir, d.num, sr_size(a->sr), row_perm, col_perm, P);
    if (s != SPGEMM_OK) {
        delete P;
        return s;
    }
    P->sr = a->sr;
    P->checked = true;
    *out = P;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_mat_transpose(spgemm_ctx_t ctx, spgemm_mat_t a, spgemm_mat_t* out) {
    if (!ctx || !a || !out) return SPGEMM_ERR_INVALID_ARG;
    if (a->fmt == SPGEMM_FMT_DCSC) return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "transpose of a DCSC handle");
    SG_TRY(check_handles(ctx, {a}));
    auto* T = new spgemm_mat();
    T->checked = true;
    spgemm_status_t s;
    if (a->fmt == SPGEMM_FMT_CSR) {
        // CSR(A) stores CSC(A^T): its arrays already are A^T in CSC; copy nothing, borrow
        T->ctx = ctx;
        T->fmt = SPGEMM_FMT_CSC;
        T->m = a->n;
        T->n = a->m;
        T->nnz = a->nnz;
        T->nzc = a->m;
        T->cp = a->cp;
        T->ir = a->ir;
        T->num = a->num;
        T->owned = a->owned;
        s = SPGEMM_OK;
    } else {
        s = transpose_csc(ctx, a->m, a->n, a->nnz, a->cp, a->ir, a->num, sr_size(a->sr), T);
    }
    if (s != SPGEMM_OK) {
        delete T;
        return s;
    }
    T->sr = a->sr;
    *out = T;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_mat_to_dcsc(spgemm_ctx_t ctx, spgemm_mat_t csc, int build_aux, spgemm_mat_t* out) {
    if (!ctx || !csc || !out) return SPGEMM_ERR_INVALID_ARG;
    if (csc->fmt != SPGEMM_FMT_CSC) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "to_dcsc expects a CSC handle");
    SG_TRY(check_handles(ctx, {csc}));
    auto* D = new spgemm_mat();
    D->checked = true;
    spgemm_status_t s = make_dcsc(ctx, csc, build_aux != 0, D);
    if (s != SPGEMM_OK) {
        delete D;
        return s;
    }
    *out = D;
    return SPGEMM_OK;
}

spgemm_status_t spgemm_mat_validate(spgemm_mat_t M) {
    if (!M) return SPGEMM_ERR_INVALID_ARG;
    spgemm_ctx* ctx = M->ctx;
    if (M->fmt == SPGEMM_FMT_DCSC) return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "validate of DCSC");
    // stored arrays: CSC with (rows = stored m) x (cols = stored n)
    const int64_t sm = M->fmt == SPGEMM_FMT_CSR ? M->n : M->m;
    const int64_t sn = M->fmt == SPGEMM_FMT_CSR ? M->m : M->n;
    auto flag = ctx_buf(ctx, 16);
    if (!flag) return set_err(ctx, SPGEMM_ERR_OOM, "validate flag");
    SG_CUDA(ctx, cudaMemsetAsync(flag->p, 0, 4, ctx->stream));
    int h = 0;
    if (sn > 0) {
        k_validate<<<grid_for(sn), 256, 0, ctx->stream>>>(M->cp, M->ir, sm, sn, M->nnz, (int*)flag->p);
        note_launch();
    } else {
        int64_t c0 = -1;
        SG_TRY(read_back(ctx, &c0, M->cp, 8));
        SG_TRY(sync_ctx(ctx));
        if (c0 != 0 || M->nnz != 0) h = 1;
    }
    if (sn > 0) {
        SG_TRY(read_back(ctx, &h, flag->p, 4));
        SG_TRY(sync_ctx(ctx));
    }
    static const char* why[] = {"", "colptr[0] != 0", "colptr[n] != nnz", "colptr not monotone",
                                "row index out of range", "rows not strictly ascending in a column"};
    if (h) return set_err(ctx, SPGEMM_ERR_BAD_FORMAT, "%s", why[h < 6 ? h : 0]);
    M->checked = true;
    return SPGEMM_OK;
}

}  // extern "C"
