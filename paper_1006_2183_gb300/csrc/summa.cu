// 2D Sparse SUMMA on a virtual g x g block grid of one GPU (Sections 3.2 and
// 3.5; the paper's own single-processor simulation of the grid is Section 5.3).
//
//   1. A and B are split into g x g blocks of ceil(dim/g) rows and columns
//      (Section 3.5: SUMMA generalises to dimensions that the grid does not
//      divide; the last block may be short or empty).  Every block is stored as
//      DCSC with the AUX column index (Section 2.3), built on the device.
//   2. Stage s multiplies A(I,s) * B(s,J) for every I, J: hypersparse block
//      products that walk the nonzero columns of B(s,J) and find A(I,s)(:,l)
//      through AUX.  All stages run as one batched execution of the column
//      kernels (or `summa_merge_every` stages at a time).
//   3. The stage partials are merged into C (Section 6.1 keeps the partial
//      triples and merges them later; Section 4.2 prices the additions).  The
//      merge is itself computed as a product: with P the matrix whose columns are
//      the partial columns and S the selector with S(u, t) = 1 when partial
//      column u belongs to output column t, C = P * S, where (x) by the
//      semiring's one is exact and (+) does the merge.  Partials keep the local
//      rows of their block row I, and the merge's output columns are
//      t = j * g + I: each merge column covers one block of mb rows, and the g
//      blocks of C(:, j) are adjacent, so C's column pointers are every g-th
//      entry of the merge's.
#include <algorithm>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>

#include "internal.cuh"

using namespace sg;

namespace {

// Block key of every entry (32-bit divisions: rows, columns and block sizes are
// below 2^31); a row outside [0, m) sets *bad and gets the key of block (0, J).
__global__ void k_block_keys(const int64_t* __restrict__ cp, const int32_t* __restrict__ ir, int64_t n, int64_t m,
                             int64_t mb, int64_t nb, int g, uint32_t* __restrict__ keys, uint32_t* __restrict__ pay,
                             unsigned long long* __restrict__ bad) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
    if (j >= n) return;
    const uint32_t J = (uint32_t)j / (uint32_t)nb;
    for (int64_t t = cp[j] + sub; t < cp[j + 1]; t += 8) {
        const int32_t r = ir[t];
        uint32_t I = 0;
        if (r < 0 || (int64_t)r >= m) atomicAdd(bad, 1ull);
        else I = (uint32_t)r / (uint32_t)mb;
        keys[t] = J * (uint32_t)g + I;   // block (I, J), column-block major
        pay[t] = (uint32_t)t;
    }
}

__global__ void k_block_colid(const int64_t* __restrict__ cp, int64_t n, int32_t* __restrict__ col) {
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const int sub = threadIdx.x & 7;
    if (j >= n) return;
    for (int64_t t = cp[j] + sub; t < cp[j + 1]; t += 8) col[t] = (int32_t)j;
}

// Gather into block order, local indices; DCSC column-start flags; per-block counts.
template <int W>
__global__ void k_block_gather(const uint32_t* __restrict__ skey, const uint32_t* __restrict__ perm, int64_t nnz,
                               const int32_t* __restrict__ ir, const int32_t* __restrict__ colid,
                               const void* __restrict__ num, int64_t mb, int64_t nb, int g, int32_t* __restrict__ lir,
                               int32_t* __restrict__ lcol, void* __restrict__ lnum, int64_t* __restrict__ flag) {
    using Wt = typename std::conditional<W == 1, uint8_t, typename std::conditional<W == 4, uint32_t, uint64_t>::type>::type;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = skey[t];
        const uint32_t src = perm[t];
        const int64_t I = key % (uint32_t)g, J = key / (uint32_t)g;
        const int32_t c = colid[src];
        lir[t] = (int32_t)(ir[src] - I * mb);
        const int32_t lc = (int32_t)(c - J * nb);
        lcol[t] = lc;
        if (num) reinterpret_cast<Wt*>(lnum)[t] = reinterpret_cast<const Wt*>(num)[src];
        flag[t] = t == 0 || skey[t - 1] != key || colid[perm[t - 1]] != c;
    }
}

// Entries and nonzero columns per block from the sorted keys: block b holds the
// keys in [lower_bound(b), lower_bound(b + 1)), its column starts are the flags
// there (pos = exclusive scan of the flags, nnz + 1 entries).
__global__ void k_block_counts(const uint32_t* __restrict__ skey, int64_t nnz, const int64_t* __restrict__ pos,
                               int nblk, unsigned long long* __restrict__ bnnz, unsigned long long* __restrict__ bnzc) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nblk) return;
    auto lb = [&](uint32_t key) {
        int64_t lo = 0, hi = nnz;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (skey[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    const int64_t lo = lb((uint32_t)b), hi = lb((uint32_t)b + 1);
    bnnz[b] = (unsigned long long)(hi - lo);
    bnzc[b] = (unsigned long long)(pos[hi] - pos[lo]);
}

__global__ void k_block_dcsc(const uint32_t* __restrict__ skey, const int32_t* __restrict__ lcol,
                             const int64_t* __restrict__ flag, const int64_t* __restrict__ pos, int64_t nnz,
                             int32_t* __restrict__ jc, int64_t* __restrict__ dcp) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * blockDim.x) {
        if (flag[t]) {
            const int64_t q = pos[t];
            jc[q] = lcol[t];
            dcp[q + skey[t]] = t;   // block b's CP array is shifted by b for its end slot
        }
    }
}

// One CTA per block: end slot of CP and the AUX index.
__global__ void k_block_aux(int nblk, const int64_t* __restrict__ boff, const int64_t* __restrict__ jcbase,
                            const int64_t* __restrict__ auxbase, const int64_t* __restrict__ chunk,
                            const int64_t* __restrict__ naux, const int32_t* __restrict__ jc, int64_t* __restrict__ dcp,
                            int32_t* __restrict__ aux) {
    const int b = blockIdx.x;
    if (b >= nblk) return;
    const int64_t nzc = jcbase[b + 1] - jcbase[b];
    if (threadIdx.x == 0) dcp[jcbase[b] + b + nzc] = boff[b + 1];
    const int32_t* bj = jc + jcbase[b];
    int32_t* ba = aux + auxbase[b];
    const int64_t na = naux[b], ch = chunk[b];
    for (int64_t t = threadIdx.x; t <= na; t += blockDim.x) {
        if (t == na) {
            ba[t] = (int32_t)nzc;
            continue;
        }
        int64_t v = t * ch, lo = 0, hi = nzc;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if ((int64_t)bj[mid] < v) lo = mid + 1;
            else hi = mid;
        }
        ba[t] = (int32_t)lo;
    }
}

// Output column of every item: col_base + JC[p] of the product's B.
__global__ void k_item_outcol(Items it, const int32_t* __restrict__ item_prod, int g, uint32_t* __restrict__ oc,
                              int64_t ofs) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < it.nitems; u += (int64_t)gridDim.x * blockDim.x) {
        const int prod = item_prod[u];
        const Prod* pr = it.prods + prod;
        const int64_t p = u - it.item_base[prod];
        const int64_t j = pr->B.jc ? pr->B.jc[p] : p;
        oc[ofs + u] = (uint32_t)((pr->col_base + j) * g + pr->blk);
    }
}

__global__ void k_iota_cols(uint32_t* oc, int64_t n) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        oc[j] = (uint32_t)j;
}

// The selector's rows for one run of merge inputs [u0, u0 + cnt) whose output columns
// oc[u] are all different (the accumulated columns, or the partial columns of one
// stage): each input takes the next free slot of its column.  The runs are filled in
// input order, one launch after another, so every column lists its inputs in input
// order, the order a stable sort by output column gives.
__global__ void k_sel_fill(const uint32_t* __restrict__ oc, int64_t u0, int64_t cnt, int64_t* __restrict__ cur,
                           int32_t* __restrict__ sir) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = u0 + i;
        const uint32_t t = oc[u];
        const int64_t pos = cur[t];
        sir[pos] = (int32_t)u;
        cur[t] = pos + 1;
    }
}

// C's column pointers from the merge's: cp[j] = Coff[j * g], j = 0..n.
__global__ void k_every_gth(const int64_t* __restrict__ Coff, int64_t n, int g, int64_t* __restrict__ cp) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= n; j += (int64_t)gridDim.x * blockDim.x)
        cp[j] = Coff[j * g];
}

__global__ void k_hist_u32(const uint32_t* __restrict__ k, int64_t n, int64_t* __restrict__ cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(reinterpret_cast<unsigned long long*>(cnt + k[i]), 1ull);
}

__global__ void k_add_offset(const int64_t* __restrict__ in, int64_t n, int64_t add, int64_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] + add;
}

// Flops per product: the items of a product are contiguous, so each thread sums
// a run of PF_RUN items and adds once per product it meets.
constexpr int PF_RUN = 32;
__global__ void k_prod_flops(Items it, const int32_t* __restrict__ item_prod, const int64_t* __restrict__ flops,
                             unsigned long long* __restrict__ pf) {
    const int64_t nrun = (it.nitems + PF_RUN - 1) / PF_RUN;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nrun; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u0 = c * PF_RUN, u1 = u0 + PF_RUN < it.nitems ? u0 + PF_RUN : it.nitems;
        int cur = item_prod[u0];
        unsigned long long acc = 0;
        for (int64_t u = u0; u < u1; ++u) {
            const int p = item_prod[u];
            if (p != cur) {
                if (acc) atomicAdd(pf + cur, acc);
                cur = p;
                acc = 0;
            }
            acc += (unsigned long long)flops[u];
        }
        if (acc) atomicAdd(pf + cur, acc);
    }
}

int gridn(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div64(n, 256), sm_count() * 32)); }

// A matrix split into g x g DCSC+AUX blocks (all blocks share the arrays).
struct Blocked {
    int g = 0;
    int64_t m = 0, n = 0, mb = 0, nb = 0;
    std::vector<DMat> blk;   // blk[J * g + I]
    std::vector<std::shared_ptr<DevBuf>> bufs;
    const DMat& at(int I, int J) const { return blk[(size_t)J * g + I]; }
};

// Two operands that are the same stored matrix (same arrays and shape).
bool same_arrays(const DMat& a, const DMat& b) {
    return a.m == b.m && a.n == b.n && a.nnz == b.nnz && a.cp == b.cp && a.ir == b.ir && a.num == b.num &&
           a.jc == b.jc;
}

spgemm_status_t partition(spgemm_ctx* ctx, const DMat& M, size_t w, int g, Blocked* out) {
    cudaStream_t st = ctx->stream;
    const int64_t m = M.m, n = M.n, nnz = M.nnz;
    const int64_t mb = std::max<int64_t>(1, ceil_div64(m, g)), nb = std::max<int64_t>(1, ceil_div64(n, g));
    const int nblk = g * g;
    out->g = g;
    out->m = m;
    out->n = n;
    out->mb = mb;
    out->nb = nb;
    if (nnz > (int64_t)UINT32_MAX) return set_err(ctx, SPGEMM_ERR_INDEX_OVERFLOW, "partition: nnz beyond 2^32");
    const int64_t nz1 = std::max<int64_t>(nnz, 1);
    // owned arrays of the blocks
    auto irb = ctx_buf(ctx, 4 * nz1);
    auto vb = ctx_buf(ctx, w * nz1);
    auto jcb = ctx_buf(ctx, 4 * nz1);
    auto cpb = ctx_buf(ctx, 8 * (nz1 + nblk + 1));
    if (!irb || !vb || !jcb || !cpb) return set_err(ctx, SPGEMM_ERR_OOM, "partition arrays");
    // temporaries
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    size_t o_k0 = take(4 * nz1), o_v0 = take(4 * nz1), o_k1 = take(4 * nz1), o_v1 = take(4 * nz1);
    size_t o_col = take(4 * nz1), o_lcol = take(4 * nz1), o_flag = take(8 * nz1), o_pos = take(8 * (nz1 + 1));
    size_t o_cnt = take(8 * (2 * nblk + 1));
    size_t o_rs = take(radix_tmp_bytes(nz1)), o_sc = take(scan_tmp_bytes(std::max<int64_t>(nz1, nblk)));
    auto tmp = ctx_buf(ctx, off);
    if (!tmp) return set_err(ctx, SPGEMM_ERR_OOM, "partition temporaries");
    char* t = (char*)tmp->p;
    uint32_t *k0 = (uint32_t*)(t + o_k0), *v0 = (uint32_t*)(t + o_v0), *k1 = (uint32_t*)(t + o_k1),
             *v1 = (uint32_t*)(t + o_v1);
    int32_t* colid = (int32_t*)(t + o_col);
    int32_t* lcol = (int32_t*)(t + o_lcol);
    int64_t* flag = (int64_t*)(t + o_flag);
    int64_t* pos = (int64_t*)(t + o_pos);
    unsigned long long* bcnt = (unsigned long long*)(t + o_cnt);   // bnnz[nblk], bnzc[nblk], bad rows
    SG_CUDA(ctx, cudaMemsetAsync(bcnt, 0, 16 * nblk + 8, st));
    std::vector<int64_t> hnnz(nblk, 0), hnzc(nblk, 0);
    if (nnz > 0) {
        k_block_keys<<<(int)ceil_div64(n * 8, 256) + 1, 256, 0, st>>>(M.cp, M.ir, n, m, mb, nb, g, k0, v0,
                                                                        bcnt + 2 * nblk);
        k_block_colid<<<(int)ceil_div64(n * 8, 256) + 1, 256, 0, st>>>(M.cp, n, colid);
        note_launch(2);
        int bits = 0;
        while (bits < 32 && (int64_t(1) << bits) < nblk) ++bits;
        bool second = false;
        radix_sort_pairs(st, k0, v0, k1, v1, nnz, bits, t + o_rs, &second);
        uint32_t* sk = second ? k1 : k0;
        uint32_t* sp = second ? v1 : v0;
        switch (w) {
        case 1: k_block_gather<1><<<gridn(nnz), 256, 0, st>>>(sk, sp, nnz, M.ir, colid, M.num, mb, nb, g, (int32_t*)irb->p, lcol, vb->p, flag); break;
        case 4: k_block_gather<4><<<gridn(nnz), 256, 0, st>>>(sk, sp, nnz, M.ir, colid, M.num, mb, nb, g, (int32_t*)irb->p, lcol, vb->p, flag); break;
        default: k_block_gather<8><<<gridn(nnz), 256, 0, st>>>(sk, sp, nnz, M.ir, colid, M.num, mb, nb, g, (int32_t*)irb->p, lcol, vb->p, flag); break;
        }
        note_launch();
        launch_exclusive_scan(st, flag, nnz, pos, t + o_sc);
        k_block_dcsc<<<gridn(nnz), 256, 0, st>>>(sk, lcol, flag, pos, nnz, (int32_t*)jcb->p, (int64_t*)cpb->p);
        k_block_counts<<<(int)ceil_div64(nblk, 256), 256, 0, st>>>(sk, nnz, pos, nblk, bcnt, bcnt + nblk);
        note_launch(2);
        std::vector<unsigned long long> hc(2 * nblk + 1);
        SG_TRY(read_back(ctx, hc.data(), bcnt, 16 * nblk + 8));
        SG_TRY(sync_ctx(ctx));
        if (hc[2 * nblk])
            return set_err(ctx, SPGEMM_ERR_BAD_FORMAT, "partition: %llu row indices outside [0, %lld)",
                           (unsigned long long)hc[2 * nblk], (long long)m);
        for (int b = 0; b < nblk; ++b) {
            hnnz[b] = (int64_t)hc[b];
            hnzc[b] = (int64_t)hc[nblk + b];
        }
    }
    // per-block layout on the host
    std::vector<int64_t> hboff(nblk + 1, 0), hjcb(nblk + 1, 0), hauxb(nblk + 1, 0), hchunk(nblk, 1), hnaux(nblk, 0);
    for (int b = 0; b < nblk; ++b) {
        const int I = b % g, J = b / g;
        (void)I;
        const int64_t ncols = std::max<int64_t>(0, std::min<int64_t>(nb, n - (int64_t)J * nb));
        hboff[b + 1] = hboff[b] + hnnz[b];
        hjcb[b + 1] = hjcb[b] + hnzc[b];
        hchunk[b] = hnzc[b] > 0 ? ceil_div64(ncols, hnzc[b]) : std::max<int64_t>(ncols, 1);
        hnaux[b] = ncols > 0 ? ceil_div64(ncols, hchunk[b]) : 0;
        hauxb[b + 1] = hauxb[b] + hnaux[b] + 1;
    }
    auto auxb = ctx_buf(ctx, 4 * std::max<int64_t>(hauxb[nblk], 1));
    auto meta = ctx_buf(ctx, 8 * (4 * (nblk + 1) + nblk));
    if (!auxb || !meta) return set_err(ctx, SPGEMM_ERR_OOM, "aux arrays");
    int64_t* dm = (int64_t*)meta->p;
    std::vector<int64_t> hm;
    hm.insert(hm.end(), hboff.begin(), hboff.end());
    hm.insert(hm.end(), hjcb.begin(), hjcb.end());
    hm.insert(hm.end(), hauxb.begin(), hauxb.end());
    hm.insert(hm.end(), hchunk.begin(), hchunk.end());
    hm.insert(hm.end(), hnaux.begin(), hnaux.end());
    hm.push_back(0);
    SG_CUDA(ctx, cudaMemcpyAsync(dm, hm.data(), 8 * hm.size(), cudaMemcpyHostToDevice, st));
    k_block_aux<<<nblk, 128, 0, st>>>(nblk, dm, dm + (nblk + 1), dm + 2 * (nblk + 1), dm + 3 * (nblk + 1),
                                      dm + 3 * (nblk + 1) + nblk, (const int32_t*)jcb->p, (int64_t*)cpb->p,
                                      (int32_t*)auxb->p);
    note_launch();
    SG_TRY(sync_ctx(ctx));   // host vectors above are copied before they go out of scope
    out->blk.assign(nblk, DMat());
    for (int b = 0; b < nblk; ++b) {
        const int I = b % g, J = b / g;
        DMat d;
        d.m = std::max<int64_t>(0, std::min<int64_t>(mb, m - (int64_t)I * mb));
        d.n = std::max<int64_t>(0, std::min<int64_t>(nb, n - (int64_t)J * nb));
        d.nzc = hnzc[b];
        d.nnz = hnnz[b];
        d.cp = (const int64_t*)cpb->p + hjcb[b] + b;
        d.jc = (const int32_t*)jcb->p + hjcb[b];
        d.aux = (const int32_t*)auxb->p + hauxb[b];
        d.chunk = hchunk[b];
        d.naux = hnaux[b];
        d.ir = (const int32_t*)irb->p;
        d.num = M.num ? vb->p : nullptr;
        out->blk[b] = d;
    }
    out->bufs = {irb, vb, jcb, cpb, auxb};
    return SPGEMM_OK;
}

// C (m x n) = merge of `ncols` sorted partial columns: column u of P (rows
// global, colptr Pcp) is added into output column oc[u].
// Stage partials go to upper-bound slots (no count pass) below this many slots.
// Stage partials go to upper-bound slots (no count pass) when those slots, their
// rows and values, take at most this share of the free device memory (the merge
// that reads them needs about as much again).
constexpr double BOUNDED_MEM_SHARE = 0.45;

bool bounded_fits(const Engine& E) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const double bytes = (double)E.flops_total * (4.0 + (double)sr_size(E.sr)) + 24.0 * (double)E.it.nitems;
    return bytes <= BOUNDED_MEM_SHARE * (double)free_b;
}

// Merges the partial columns P (local rows < mb; column u goes to merge column
// oc[u] = j * g + I) into the mb x (n g) matrix of merge columns, or, when
// `final`, into C (m x n, global rows I * mb + local row).  `runs` cover [0, ncols)
// in order, each a range of inputs whose merge columns are all different.
spgemm_status_t merge_columns(spgemm_ctx* ctx, spgemm_semiring_t sr, const spgemm_opts_t& opts, int64_t m,
                              int64_t mb, int64_t n0, int g, bool final, int64_t ncols, const int64_t* Pcp,
                              const int64_t* Pce, const int32_t* Pir, const void* Pv, int64_t pnnz,
                              const uint32_t* oc, const std::vector<std::pair<int64_t, int64_t>>& runs,
                              spgemm_mat_t* C) {
    cudaStream_t st = ctx->stream;
    PhaseTimer tm(ctx, SPGEMM_PHASE_MERGE, sr);
    const int64_t n = n0 * g;   // merge columns
    const int64_t nc1 = std::max<int64_t>(ncols, 1);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    size_t o_cnt = take(8 * (n + 1)), o_sc = take(scan_tmp_bytes(std::max<int64_t>(n, 1)));
    auto tmp = ctx_buf(ctx, off);
    auto scp = ctx_buf(ctx, 8 * (n + 1));
    auto sir = ctx_buf(ctx, 4 * nc1);
    if (!tmp || !scp || !sir) return set_err(ctx, SPGEMM_ERR_OOM, "merge selector");
    char* t = (char*)tmp->p;
    // the selector S in CSC: inputs per merge column (a count and a scan), then every
    // input placed at the next free slot of its column, run after run
    int64_t* cnt = (int64_t*)(t + o_cnt);
    SG_CUDA(ctx, cudaMemsetAsync(cnt, 0, 8 * (n + 1), st));
    if (ncols > 0) {
        k_hist_u32<<<gridn(ncols), 256, 0, st>>>(oc, ncols, cnt);
        note_launch();
    }
    launch_exclusive_scan(st, cnt, n, (int64_t*)scp->p, t + o_sc);
    if (ncols > 0) {
        SG_CUDA(ctx, cudaMemcpyAsync(cnt, scp->p, 8 * n, cudaMemcpyDeviceToDevice, st));
        for (const auto& r : runs) {
            if (r.second <= r.first) continue;
            k_sel_fill<<<gridn(r.second - r.first), 256, 0, st>>>(oc, r.first, r.second - r.first, cnt,
                                                                  (int32_t*)sir->p);
            note_launch();
        }
    }
    // C = P * S
    Prod pr;
    pr.A = csc_view(mb, ncols, pnnz, Pcp, Pir, Pv);
    pr.A.ce = Pce;   // partials written into bounded slots: column u ends at Pce[u]
    pr.B = csc_view(ncols, n, ncols, (const int64_t*)scp->p, (const int32_t*)sir->p, nullptr);
    if (final) {
        pr.rb_cycle = g;
        pr.rb_step = (int32_t)mb;
    }
    Engine E;
    struct Quiet {   // the merge's own phases are reported as one MERGE phase
        spgemm_ctx* c;
        explicit Quiet(spgemm_ctx* x) : c(x) { ++c->timing_quiet; }
        ~Quiet() { --c->timing_quiet; }
    } quiet(ctx);
    SG_TRY(engine_setup(&E, ctx, sr, opts, {pr}, false));
    SG_TRY(engine_symbolic(&E));
    std::shared_ptr<DevBuf> rbuf, vbuf;
    SG_TRY(engine_alloc_out(&E, &rbuf, &vbuf));
    SG_TRY(engine_numeric(&E, (int32_t*)rbuf->p, vbuf->p));
    if (!final) {
        *C = new_owned_csc(ctx, sr, mb, n, E.nnz_total, {E.Coff_buf, rbuf, vbuf}, E.Coff, (const int32_t*)rbuf->p,
                           vbuf->p);
        return SPGEMM_OK;
    }
    auto cp = ctx_buf(ctx, 8 * (n0 + 1));
    if (!cp) return set_err(ctx, SPGEMM_ERR_OOM, "merge column pointers");
    k_every_gth<<<gridn(n0 + 1), 256, 0, st>>>(E.Coff, n0, g, (int64_t*)cp->p);
    note_launch();
    *C = new_owned_csc(ctx, sr, m, n0, E.nnz_total, {cp, rbuf, vbuf}, (const int64_t*)cp->p, (const int32_t*)rbuf->p,
                       vbuf->p);
    return SPGEMM_OK;
}

// One group of stages, multiplied and ready to merge.
struct Group {
    Engine E;
    std::shared_ptr<DevBuf> rbuf, vbuf, colbuf;
    const int64_t* pstart = nullptr;   // partial columns with gaps (bounded slots), or null
    const int64_t* pend = nullptr;
    int64_t U = 0, pn = 0;             // partial columns, partial entries
    bool final = false;                // the last group: its merge writes C
    cudaEvent_t ready = nullptr;       // recorded after the products (pipelined mode)
};

// Stage products A(I,s) * B(s,J) of one group, on ctx's stream (stage-major items).
spgemm_status_t stage_products(spgemm_ctx* ctx, spgemm_semiring_t sr, const spgemm_opts_t& o,
                               const std::vector<Prod>& grp, bool single_merge, Group* G) {
    if (grp.empty()) return SPGEMM_OK;
    Engine& E = G->E;
    SG_TRY(engine_setup(&E, ctx, sr, o, grp, false));
    if (o.block_kernel == 1) {
        SG_TRY(engine_esc(&E, &G->rbuf, &G->vbuf));   // outer-product order, Section 2.4
    } else if (single_merge && bounded_fits(E)) {
        // one merge reads the partials where they were written: no count pass for them
        SG_TRY(engine_numeric_bounded(&E, &G->rbuf, &G->vbuf, &G->colbuf, &G->pstart, &G->pend));
    } else {
        SG_TRY(engine_symbolic(&E));
        SG_TRY(engine_alloc_out(&E, &G->rbuf, &G->vbuf));
        SG_TRY(engine_numeric(&E, (int32_t*)G->rbuf->p, G->vbuf->p));
    }
    G->U = E.it.nitems;
    G->pn = E.nnz_total;
    // stage flops for the statistics
    auto pf = ctx_buf(ctx, 8 * grp.size());
    if (!pf) return set_err(ctx, SPGEMM_ERR_OOM, "stage flops");
    SG_CUDA(ctx, cudaMemsetAsync(pf->p, 0, 8 * grp.size(), ctx->stream));
    k_prod_flops<<<gridn(ceil_div64(G->U, PF_RUN)), 256, 0, ctx->stream>>>(E.it, E.item_prod, E.flops, (unsigned long long*)pf->p);
    note_launch();
    std::vector<unsigned long long> hpf(grp.size());
    SG_TRY(read_back(ctx, hpf.data(), pf->p, 8 * grp.size()));
    SG_TRY(sync_ctx(ctx));
    for (size_t i = 0; i < grp.size(); ++i) ctx->summa_stage_flops[grp[i].tag] += (int64_t)hpf[i];
    return SPGEMM_OK;
}

// Merges the group's partials with the accumulated merge columns `acc` (null
// before the first merge), on mctx's stream and through mctx's allocator.
spgemm_status_t merge_group(spgemm_ctx* mctx, spgemm_semiring_t sr, const spgemm_opts_t& o, int64_t m, int64_t mb,
                            int64_t n, int g, Group& G, spgemm_mat_t acc, spgemm_mat_t* Cn) {
    const size_t w = sr_size(sr);
    const int64_t U = G.U, pn = G.pn;
    const Engine& E = G.E;
    // columns to merge: the accumulated C (if any) followed by this group's partial columns
    const int64_t nacc = acc ? n * g : 0;   // merge columns so far
    const int64_t accnz = acc ? acc->nnz : 0;
    const int64_t ncols = nacc + U;
    const int64_t pnz = accnz + pn;
    cudaStream_t stq = mctx->stream;
    auto ocb = ctx_buf(mctx, 4 * std::max<int64_t>(ncols, 1));
    if (!ocb) return set_err(mctx, SPGEMM_ERR_OOM, "merge keys");
    uint32_t* oc = (uint32_t*)ocb->p;
    std::shared_ptr<DevBuf> pcp, pir, pv;
    const int64_t* Pcp;
    const int32_t* Pir;
    const void* Pv;
    const int64_t* Pce = nullptr;
    if (!acc && U > 0) {
        // the partials alone: merge them in place
        Pcp = G.pstart ? G.pstart : E.Coff;
        Pce = G.pend;
        Pir = (const int32_t*)G.rbuf->p;
        Pv = G.vbuf->p;
    } else {
        pcp = ctx_buf(mctx, 8 * (ncols + 1));
        pir = ctx_buf(mctx, 4 * std::max<int64_t>(pnz, 1));
        pv = ctx_buf(mctx, w * std::max<int64_t>(pnz, 1));
        if (!pcp || !pir || !pv) return set_err(mctx, SPGEMM_ERR_OOM, "merge inputs");
        if (acc) {
            SG_CUDA(mctx, cudaMemcpyAsync(pcp->p, acc->cp, 8 * nacc, cudaMemcpyDeviceToDevice, stq));
            if (accnz) {
                SG_CUDA(mctx, cudaMemcpyAsync(pir->p, acc->ir, 4 * accnz, cudaMemcpyDeviceToDevice, stq));
                SG_CUDA(mctx, cudaMemcpyAsync(pv->p, acc->num, w * accnz, cudaMemcpyDeviceToDevice, stq));
            }
        }
        if (U > 0) {
            k_add_offset<<<gridn(U + 1), 256, 0, stq>>>(E.Coff, U + 1, accnz, (int64_t*)pcp->p + nacc);
            note_launch();
            if (pn) {
                SG_CUDA(mctx, cudaMemcpyAsync((int32_t*)pir->p + accnz, G.rbuf->p, 4 * pn, cudaMemcpyDeviceToDevice, stq));
                SG_CUDA(mctx, cudaMemcpyAsync((char*)pv->p + w * accnz, G.vbuf->p, w * pn, cudaMemcpyDeviceToDevice, stq));
            }
        } else if (acc) {
            SG_CUDA(mctx, cudaMemcpyAsync((int64_t*)pcp->p + nacc, acc->cp + nacc, 8, cudaMemcpyDeviceToDevice, stq));
        } else {
            SG_CUDA(mctx, cudaMemsetAsync(pcp->p, 0, 8, stq));
        }
        Pcp = (const int64_t*)pcp->p;
        Pir = (const int32_t*)pir->p;
        Pv = pv->p;
    }
    // runs of inputs whose merge columns differ: the accumulated columns, then the
    // partial columns of each stage (one per merge column at most; items are stage-major)
    std::vector<std::pair<int64_t, int64_t>> runs;
    if (acc) {
        k_iota_cols<<<gridn(nacc), 256, 0, stq>>>(oc, nacc);
        note_launch();
        runs.push_back({0, nacc});
    }
    if (U > 0) {
        k_item_outcol<<<gridn(U), 256, 0, stq>>>(E.it, E.item_prod, g, oc, nacc);
        note_launch();
        for (size_t i = 0; i < E.hprods.size();) {
            size_t j = i;
            while (j < E.hprods.size() && E.hprods[j].tag == E.hprods[i].tag) ++j;
            runs.push_back({nacc + E.hitem_base[i], nacc + E.hitem_base[j]});
            i = j;
        }
    }
    return merge_columns(mctx, sr, o, m, mb, n, g, G.final, ncols, Pcp, Pce, Pir, Pv, pnz, oc, runs, Cn);
}

// Hand-over between the products (calling thread, ctx's stream) and the merges
// (worker thread, merge context's stream) of the two-stream pipeline.
struct Pipe {
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::unique_ptr<Group>> todo;   // multiplied, not merged
    std::deque<std::unique_ptr<Group>> done;   // merged: freed by the calling thread
    bool closed = false;                       // no more groups will come
    bool abort = false;                        // the products failed: merge nothing more
    spgemm_status_t status = SPGEMM_OK;        // the worker's (read after join)
    spgemm_mat_t result = nullptr;             // C, after the final group's merge
};

void merge_worker(Pipe* P, spgemm_ctx* mctx, spgemm_semiring_t sr, spgemm_opts_t o, int64_t m, int64_t mb,
                  int64_t n, int g) {
    cudaSetDevice(mctx->device);
    spgemm_mat_t acc = nullptr;
    std::unique_ptr<spgemm_mat> hold;
    for (;;) {
        std::unique_ptr<Group> G;
        bool abort;
        {
            std::unique_lock<std::mutex> lk(P->mu);
            P->cv.wait(lk, [&] { return !P->todo.empty() || P->closed; });
            if (P->todo.empty()) break;   // closed and drained
            G = std::move(P->todo.front());
            P->todo.pop_front();
            abort = P->abort;
        }
        if (P->status == SPGEMM_OK && !abort) {
            spgemm_status_t s = SPGEMM_OK;
            cudaError_t e = cudaStreamWaitEvent(mctx->stream, G->ready, 0);
            if (e != cudaSuccess) s = check_cuda(mctx, e, "wait for the stage products at " SG_WHERE);
            spgemm_mat_t Cn = nullptr;
            if (s == SPGEMM_OK) s = merge_group(mctx, sr, o, m, mb, n, g, *G, acc, &Cn);
            if (s == SPGEMM_OK) {
                hold.reset(Cn);
                acc = Cn;
                if (G->final) P->result = hold.release();
            }
            P->status = s;
        }
        // the merge no longer reads the group's arrays once its stream is drained
        cudaError_t e = cudaStreamSynchronize(mctx->stream);
        if (e != cudaSuccess && P->status == SPGEMM_OK) P->status = check_cuda(mctx, e, "merge stream at " SG_WHERE);
        cudaEventDestroy(G->ready);
        G->ready = nullptr;
        std::lock_guard<std::mutex> lk(P->mu);
        P->done.push_back(std::move(G));
    }
}

// Common driver of spgemm_summa_blocked (mctx null: one stream) and
// spgemm_summa_pipelined (merges on mctx's stream, overlapping the next
// group's stage products; Sections 7.2-7.3 overlap the stage broadcasts with
// the local work, which on one GPU becomes this stage/merge overlap).
spgemm_status_t summa_run(spgemm_ctx_t ctx, spgemm_ctx_t mctx, spgemm_mat_t A, spgemm_mat_t B, int g,
                          spgemm_semiring_t sr, const spgemm_opts_t* opts, spgemm_mat_t* C) {
    if (!ctx || !A || !B || !C) return SPGEMM_ERR_INVALID_ARG;
    if (g < 1 || g > 1024) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "grid size g = %d outside [1, 1024]", g);
    if ((int)sr < 0 || (int)sr > 3) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "bad semiring");
    if (A->sr != sr || B->sr != sr) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "operand semiring differs");
    if (A->n != B->m) return set_err(ctx, SPGEMM_ERR_DIM_MISMATCH, "inner dimensions differ");
    if (A->fmt == SPGEMM_FMT_DCSC || B->fmt == SPGEMM_FMT_DCSC)
        return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "summa takes CSC or CSR operands");
    spgemm_opts_t o;
    spgemm_opts_default(&o);
    if (opts) o = *opts;
    if (o.summa_fused != 0) return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "summa_fused is reserved (must be 0)");
    if (o.block_kernel != 0 && o.block_kernel != 1)
        return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "block_kernel %d: 0 (column tiers) or 1 (expand-sort-compress)",
                       o.block_kernel);
    if (o.check_inputs) SG_TRY(check_handles(ctx, {A, B}));
    // boolean: whether the two operands store a false value, checked once for every stage
    // product and merge of this call (their values all come from A and B)
    struct HintGuard {
        spgemm_ctx *c, *mc;
        ~HintGuard() {
            c->bool_hint = -1;
            if (mc) mc->bool_hint = -1;
        }
    } hint_guard{ctx, mctx};
    if (sr == SPGEMM_OR_AND_BOOL) {
        auto fb = ctx_buf(ctx, 16);
        if (!fb) return set_err(ctx, SPGEMM_ERR_OOM, "false-value flag");
        SG_CUDA(ctx, cudaMemsetAsync(fb->p, 0, 4, ctx->stream));
        launch_any_false(ctx->stream, A->num, A->nnz, (int*)fb->p);
        launch_any_false(ctx->stream, B->num, B->nnz, (int*)fb->p);
        int hf = 0;
        SG_TRY(read_back(ctx, &hf, fb->p, 4));
        SG_TRY(sync_ctx(ctx));
        ctx->bool_hint = hf ? 1 : 0;
        if (mctx) mctx->bool_hint = ctx->bool_hint;
    }
    spgemm_mat_t Ac = nullptr, Bc = nullptr;
    DMat dA, dB;
    SG_TRY(to_csc_operand(ctx, A, &Ac, &dA));
    spgemm_status_t s = to_csc_operand(ctx, B, &Bc, &dB);
    std::unique_ptr<spgemm_mat> holdA(Ac), holdB(Bc);
    if (s != SPGEMM_OK) return s;
    const size_t w = sr_size(sr);
    const int64_t m = dA.m, n = dB.n;
    if (n * g >= (int64_t(1) << 32))
        return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "n * g = %lld merge columns exceed 2^32", (long long)(n * g));
    Blocked bA, bB;
    {
        PhaseTimer tp(ctx, SPGEMM_PHASE_ANALYZE, sr);
        SG_TRY(partition(ctx, dA, w, g, &bA));
        // the same matrix on both sides (A*A): one split serves as A's and as B's blocks
        if (same_arrays(dA, dB)) bB = bA;
        else SG_TRY(partition(ctx, dB, w, g, &bB));
    }
    // stage products A(I,s) * B(s,J), stage-major
    std::vector<Prod> all;
    for (int st = 0; st < g; ++st)
        for (int J = 0; J < g; ++J)
            for (int I = 0; I < g; ++I) {
                const DMat& a = bA.at(I, st);
                const DMat& b = bB.at(st, J);
                if (a.nnz == 0 || b.nnz == 0 || a.m == 0 || b.n == 0) continue;
                Prod pr;
                pr.A = a;
                pr.B = b;
                pr.row_base = 0;   // local rows; the merge adds I * mb
                pr.col_base = (int64_t)J * bB.nb;
                pr.tag = st;
                pr.blk = I;
                all.push_back(pr);
            }
    ctx->summa_stage_flops.assign(g, 0);
    ctx->summa_nonempty = (int64_t)all.size();
    const int every = o.summa_merge_every > 0 ? std::min(o.summa_merge_every, g) : g;
    auto group_of = [&](int s0) {
        std::vector<Prod> grp;
        for (auto& pr : all)
            if (pr.tag >= s0 && pr.tag < s0 + every) grp.push_back(pr);
        return grp;
    };
    if (!mctx) {
        spgemm_mat_t acc = nullptr;   // C merged so far
        std::unique_ptr<spgemm_mat> hold_acc;
        for (int s0 = 0; s0 < g; s0 += every) {
            Group G;
            G.final = s0 + every >= g;
            SG_TRY(stage_products(ctx, sr, o, group_of(s0), !acc && G.final, &G));
            spgemm_mat_t Cn = nullptr;
            SG_TRY(merge_group(ctx, sr, o, m, bA.mb, n, g, G, acc, &Cn));
            hold_acc.reset(Cn);
            acc = Cn;
        }
        *C = hold_acc.release();
        return SPGEMM_OK;
    }
    // two streams: group k's merge (worker) overlaps group k+1's stage products (here)
    Pipe P;
    std::thread worker(merge_worker, &P, mctx, sr, o, m, bA.mb, n, g);
    auto release_done = [&] {
        std::deque<std::unique_ptr<Group>> d;
        {
            std::lock_guard<std::mutex> lk(P.mu);
            d.swap(P.done);
        }
    };
    for (int s0 = 0; s0 < g && s == SPGEMM_OK; s0 += every) {
        auto G = std::make_unique<Group>();
        G->final = s0 + every >= g;
        s = stage_products(ctx, sr, o, group_of(s0), every >= g, G.get());
        if (s != SPGEMM_OK) break;
        cudaError_t e = cudaEventCreateWithFlags(&G->ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(G->ready, ctx->stream);
        if (e != cudaSuccess) {
            if (G->ready) cudaEventDestroy(G->ready);
            s = check_cuda(ctx, e, "stage products event at " SG_WHERE);
            break;
        }
        {
            std::lock_guard<std::mutex> lk(P.mu);
            P.todo.push_back(std::move(G));
        }
        P.cv.notify_one();
        release_done();
    }
    {
        std::lock_guard<std::mutex> lk(P.mu);
        P.closed = true;
        P.abort = s != SPGEMM_OK;
    }
    P.cv.notify_one();
    worker.join();
    release_done();
    std::unique_ptr<spgemm_mat> result(P.result);
    if (s != SPGEMM_OK) return s;
    if (P.status != SPGEMM_OK) return set_err(ctx, P.status, "pipelined merge: %s", mctx->err.c_str());
    if (!result) return set_err(ctx, SPGEMM_ERR_CUDA, "pipelined merge produced no result");
    *C = result.release();
    return SPGEMM_OK;
}

}  // namespace

extern "C" {

spgemm_status_t spgemm_summa_blocked(spgemm_ctx_t ctx, spgemm_mat_t A, spgemm_mat_t B, int g, spgemm_semiring_t sr,
                                     const spgemm_opts_t* opts, spgemm_mat_t* C) {
    return summa_run(ctx, nullptr, A, B, g, sr, opts, C);
}

spgemm_status_t spgemm_summa_pipelined(spgemm_ctx_t ctx, spgemm_ctx_t merge_ctx, spgemm_mat_t A, spgemm_mat_t B,
                                       int g, spgemm_semiring_t sr, const spgemm_opts_t* opts, spgemm_mat_t* C) {
    if (!ctx || !merge_ctx) return SPGEMM_ERR_INVALID_ARG;
    if (merge_ctx == ctx) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "the merge context must be a second context");
    if (merge_ctx->device != ctx->device)
        return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "contexts on devices %d and %d", ctx->device, merge_ctx->device);
    return summa_run(ctx, merge_ctx, A, B, g, sr, opts, C);
}

spgemm_status_t spgemm_summa_block_flops(spgemm_ctx_t ctx, spgemm_mat_t A, spgemm_mat_t B, int g, int64_t* flops) {
    if (!ctx || !A || !B || !flops) return SPGEMM_ERR_INVALID_ARG;
    if (g < 1 || g > 1024) return set_err(ctx, SPGEMM_ERR_INVALID_ARG, "grid size g = %d outside [1, 1024]", g);
    if (A->n != B->m) return set_err(ctx, SPGEMM_ERR_DIM_MISMATCH, "inner dimensions differ");
    if (A->fmt == SPGEMM_FMT_DCSC || B->fmt == SPGEMM_FMT_DCSC)
        return set_err(ctx, SPGEMM_ERR_UNSUPPORTED, "summa takes CSC or CSR operands");
    SG_TRY(check_handles(ctx, {A, B}));
    spgemm_mat_t Ac = nullptr, Bc = nullptr;
    DMat dA, dB;
    SG_TRY(to_csc_operand(ctx, A, &Ac, &dA));
    spgemm_status_t st0 = to_csc_operand(ctx, B, &Bc, &dB);
    std::unique_ptr<spgemm_mat> holdA(Ac), holdB(Bc);
    if (st0 != SPGEMM_OK) return st0;
    const size_t w = sr_size(A->sr);
    Blocked bA, bB;
    SG_TRY(partition(ctx, dA, w, g, &bA));
    if (same_arrays(dA, dB)) bB = bA;
    else SG_TRY(partition(ctx, dB, w, g, &bB));
    const size_t g3 = (size_t)g * g * g;
    std::fill(flops, flops + g3, int64_t(0));
    std::vector<Prod> all;
    std::vector<size_t> slot;
    for (int st = 0; st < g; ++st)
        for (int J = 0; J < g; ++J)
            for (int I = 0; I < g; ++I) {
                const DMat& a = bA.at(I, st);
                const DMat& b = bB.at(st, J);
                if (a.nnz == 0 || b.nnz == 0 || a.m == 0 || b.n == 0) continue;
                Prod pr;
                pr.A = a;
                pr.B = b;
                all.push_back(pr);
                slot.push_back(((size_t)st * g + J) * g + I);
            }
    if (all.empty()) return SPGEMM_OK;
    spgemm_opts_t o;
    spgemm_opts_default(&o);
    Engine E;
    SG_TRY(engine_setup(&E, ctx, A->sr, o, all, false));
    auto pf = ctx_buf(ctx, 8 * all.size());
    if (!pf) return set_err(ctx, SPGEMM_ERR_OOM, "block flops");
    SG_CUDA(ctx, cudaMemsetAsync(pf->p, 0, 8 * all.size(), ctx->stream));
    k_prod_flops<<<gridn(ceil_div64(E.it.nitems, PF_RUN)), 256, 0, ctx->stream>>>(E.it, E.item_prod, E.flops, (unsigned long long*)pf->p);
    note_launch();
    std::vector<unsigned long long> h(all.size());
    SG_TRY(read_back(ctx, h.data(), pf->p, 8 * all.size()));
    SG_TRY(sync_ctx(ctx));
    for (size_t i = 0; i < all.size(); ++i) flops[slot[i]] = (int64_t)h[i];
    return SPGEMM_OK;
}

spgemm_status_t spgemm_summa_stats(spgemm_ctx_t ctx, int64_t* stage_flops, int g, int64_t* nonempty) {
    if (!ctx) return SPGEMM_ERR_INVALID_ARG;
    if (stage_flops)
        for (int s = 0; s < g; ++s)
            stage_flops[s] = s < (int)ctx->summa_stage_flops.size() ? ctx->summa_stage_flops[s] : 0;
    if (nonempty) *nonempty = ctx->summa_nonempty;
    return SPGEMM_OK;
}

}  // extern "C"
