/*
 * CPU oracle for C = A*B over a semiring -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load this library.  It shares no code with the CUDA path.
 *
 * Method: the column-by-column (Gustavson) formulation, Section 2.1 and
 * Section 4 (the classical O(flops + nnz + n) algorithm of the Introduction),
 * with a dense sparse accumulator (SPA, Section 3.3):
 *   C(:,j) = (+)_{k in B(:,j)}  A(:,k) (x) B(k,j)
 * taken in ascending k, then ascending i inside A(:,k).  The result column is
 * the sorted list of touched rows.  Structural semantics: an entry exists iff
 * some k pairs a stored A(i,k) with a stored B(k,j); entries whose value ends
 * up equal to the semiring zero are kept.
 *
 * Semirings (0-based indices, CSC with int64 column pointers, int32 rows):
 *   0 plus-times on double, summed with Neumaier's compensated summation
 *     (Neumaier 1974) so that the reference value carries almost no rounding;
 *   1 min-plus on float, candidate fl32(a + b), round to nearest, no FMA;
 *   2 or-and on uint8 (nonzero byte = true);
 *   3 plus-times on int64 with two's-complement wraparound.
 *
 * flops_j = sum_{k in B(:,j)} nnz(A(:,k))  (the "flops" count of Section 1).
 * All entry points return 0 on success and a negative code on bad input.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { SR_PT_F64 = 0, SR_MP_F32 = 1, SR_OR_BOOL = 2, SR_PT_I64 = 3 };

static int cmp_i32(const void* x, const void* y) {
    int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
    return (a > b) - (a < b);
}

static int set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) return nthreads;
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_max_threads(void) { return set_threads(0); }

/* flops_j for every column j of B. */
int oracle_flops(int64_t n, const int64_t* Acp, const int64_t* Bcp, const int32_t* Bir,
                 int64_t* flops) {
    for (int64_t j = 0; j < n; ++j) {
        int64_t f = 0;
        for (int64_t t = Bcp[j]; t < Bcp[j + 1]; ++t) {
            int32_t k = Bir[t];
            f += Acp[k + 1] - Acp[k];
        }
        flops[j] = f;
    }
    return 0;
}

/* Symbolic pass: nnz(C(:,j)) = |union over k in B(:,j) of pattern(A(:,k))|. */
int oracle_symbolic(int64_t m, const int64_t* Acp, const int32_t* Air,
                    int64_t n, const int64_t* Bcp, const int32_t* Bir,
                    int64_t* nnz, int nthreads) {
    int nt = set_threads(nthreads);
    int err = 0;
#pragma omp parallel num_threads(nt)
    {
        int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
        if (!mark) {
#pragma omp atomic write
            err = -2;
        } else {
            for (int64_t i = 0; i < m; ++i) mark[i] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t j = 0; j < n; ++j) {
                int64_t cnt = 0;
                for (int64_t t = Bcp[j]; t < Bcp[j + 1]; ++t) {
                    int32_t k = Bir[t];
                    for (int64_t s = Acp[k]; s < Acp[k + 1]; ++s) {
                        int32_t i = Air[s];
                        if (mark[i] != j) { mark[i] = j; ++cnt; }
                    }
                }
                nnz[j] = cnt;
            }
            free(mark);
        }
    }
    return err;
}

/* One output column, dense SPA with a touched-row list; rows emitted sorted. */
typedef struct {
    int64_t* mark;
    int32_t* list;
    double* sum;
    double* comp;
    float* mp;
    uint8_t* bl;
    uint64_t* iv;
} spa_t;

static void column_numeric(int sr, int64_t j, const int64_t* Acp, const int32_t* Air, const void* Aval,
                           const int64_t* Bcp, const int32_t* Bir, const void* Bval,
                           spa_t* s, int32_t* out_rows, void* out_vals) {
    int64_t len = 0;
    for (int64_t t = Bcp[j]; t < Bcp[j + 1]; ++t) {
        int32_t k = Bir[t];
        for (int64_t q = Acp[k]; q < Acp[k + 1]; ++q) {
            int32_t i = Air[q];
            int fresh = (s->mark[i] != j);
            if (fresh) { s->mark[i] = j; s->list[len++] = i; }
            switch (sr) {
            case SR_PT_F64: {
                double x = ((const double*)Aval)[q] * ((const double*)Bval)[t];
                if (fresh) { s->sum[i] = x; s->comp[i] = 0.0; }
                else {
                    double a = s->sum[i], u = a + x;
                    if (fabs(a) >= fabs(x)) s->comp[i] += (a - u) + x;
                    else s->comp[i] += (x - u) + a;
                    s->sum[i] = u;
                }
                break;
            }
            case SR_MP_F32: {
                volatile float x = ((const float*)Aval)[q] + ((const float*)Bval)[t];
                if (fresh || x < s->mp[i]) s->mp[i] = x;
                break;
            }
            case SR_OR_BOOL: {
                uint8_t x = (uint8_t)((((const uint8_t*)Aval)[q] != 0) && (((const uint8_t*)Bval)[t] != 0));
                if (fresh) s->bl[i] = x; else s->bl[i] = (uint8_t)(s->bl[i] | x);
                break;
            }
            default: {
                uint64_t x = (uint64_t)((const int64_t*)Aval)[q] * (uint64_t)((const int64_t*)Bval)[t];
                if (fresh) s->iv[i] = x; else s->iv[i] += x;
                break;
            }
            }
        }
    }
    qsort(s->list, (size_t)len, sizeof(int32_t), cmp_i32);
    for (int64_t p = 0; p < len; ++p) {
        int32_t i = s->list[p];
        out_rows[p] = i;
        switch (sr) {
        case SR_PT_F64: ((double*)out_vals)[p] = s->sum[i] + s->comp[i]; break;
        case SR_MP_F32: ((float*)out_vals)[p] = s->mp[i]; break;
        case SR_OR_BOOL: ((uint8_t*)out_vals)[p] = s->bl[i]; break;
        default: ((int64_t*)out_vals)[p] = (int64_t)s->iv[i]; break;
        }
    }
}

static size_t val_size(int sr) {
    switch (sr) {
    case SR_PT_F64: return 8;
    case SR_MP_F32: return 4;
    case SR_OR_BOOL: return 1;
    default: return 8;
    }
}

/* Numeric pass: fills C's rows and values given C's column pointers
 * (Ccp from the symbolic pass, prefix-summed).  Columns are independent,
 * so they are shared out across threads; each thread owns one SPA. */
int oracle_numeric(int sr, int64_t m, const int64_t* Acp, const int32_t* Air, const void* Aval,
                   int64_t n, const int64_t* Bcp, const int32_t* Bir, const void* Bval,
                   const int64_t* Ccp, int32_t* Cir, void* Cval, int nthreads) {
    if (sr < 0 || sr > 3) return -1;
    int nt = set_threads(nthreads);
    int err = 0;
    size_t w = val_size(sr);
#pragma omp parallel num_threads(nt)
    {
        spa_t s;
        memset(&s, 0, sizeof s);
        size_t mm = (size_t)(m > 0 ? m : 1);
        s.mark = (int64_t*)malloc(sizeof(int64_t) * mm);
        s.list = (int32_t*)malloc(sizeof(int32_t) * mm);
        if (sr == SR_PT_F64) { s.sum = (double*)malloc(8 * mm); s.comp = (double*)malloc(8 * mm); }
        if (sr == SR_MP_F32) s.mp = (float*)malloc(4 * mm);
        if (sr == SR_OR_BOOL) s.bl = (uint8_t*)malloc(mm);
        if (sr == SR_PT_I64) s.iv = (uint64_t*)malloc(8 * mm);
        int ok = s.mark && s.list && (s.sum || s.mp || s.bl || s.iv) && (sr != SR_PT_F64 || s.comp);
        if (!ok) {
#pragma omp atomic write
            err = -2;
        } else {
            for (int64_t i = 0; i < m; ++i) s.mark[i] = -1;
#pragma omp for schedule(dynamic, 64)
            for (int64_t j = 0; j < n; ++j)
                column_numeric(sr, j, Acp, Air, Aval, Bcp, Bir, Bval, &s, Cir + Ccp[j],
                               (char*)Cval + (size_t)Ccp[j] * w);
        }
        free(s.mark); free(s.list); free(s.sum); free(s.comp); free(s.mp); free(s.bl); free(s.iv);
    }
    return err;
}
