/*
 * Plain FP64 CPU oracle for one Markov Cluster (MCL) iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this code; the product path never does.
 * It shares no code with the CUDA library.
 *
 * Each function follows the paper's statement of the method (Algorithm 1
 * and the notation paragraph of Section II, "Notations used in this
 * paper") step by step, with no blocking, fusion or reordering:
 *
 *   expansion      B = A A, column by column, c_ij = sum_k a_ik a_kj
 *                  (Alg. 1, expansion), dense FP64 accumulator of length n;
 *   flops          flops_j = sum over k in inds(A_*j) of nnz(A_*k)
 *                  (Section II notation);
 *   prune          threshold + top-k (Alg. 1, Prune; Section II overview),
 *                  with the "recover to a mass fraction" reading:
 *                  sort the column by value descending (equal values: the
 *                  smaller row first), t = #{b >= theta},
 *                  m_rec = smallest m with (sum of the top m) >= p * s
 *                  where s is the column sum, keep the top
 *                  m* = min(K_rec, max(min(t, K), m_rec)) entries;
 *   inflation      Hadamard power (Alg. 1, inflation) followed by column
 *                  renormalisation (the matrix stays column stochastic,
 *                  Section II overview);
 *   chaos          chaos_j = max(0, max_i a_ij - sum_i a_ij^2) on the
 *                  normalised column; the convergence test of Alg. 1
 *                  ("while change in successive iterations") reads
 *                  max_j chaos_j.  The paper gives no formula: this is a
 *                  reading, pinned to closed forms (tests/golden/
 *                  chaos_cases.txt), parity unpinned against the paper;
 *   clusters       connected components of the final matrix's undirected
 *                  pattern (Alg. 1, return), union-find; label = smallest
 *                  vertex id of the component.
 *
 * Everything is FP64; the input values are whatever the caller passes
 * (the FP32 values of the GPU path, widened exactly, in parity tests).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double v;
    int32_t r;
} entry_t;

/* value descending, then row ascending */
static int cmp_value_desc(const void* pa, const void* pb) {
    const entry_t* a = (const entry_t*)pa;
    const entry_t* b = (const entry_t*)pb;
    if (a->v > b->v) return -1;
    if (a->v < b->v) return 1;
    return (a->r < b->r) ? -1 : (a->r > b->r);
}

static int cmp_row_asc(const void* pa, const void* pb) {
    const entry_t* a = (const entry_t*)pa;
    const entry_t* b = (const entry_t*)pb;
    return (a->r < b->r) ? -1 : (a->r > b->r);
}

/* Column j of B = A A with a dense accumulator.  Writes the structurally
 * nonzero entries (unsorted) to out, returns their count; *flops gets the
 * number of products a_ik * a_kj formed. */
static int64_t expand_column(int64_t n, const int64_t* colptr, const int32_t* rowidx,
                             const double* val, int64_t j, double* acc, unsigned char* seen,
                             entry_t* out, int64_t* flops) {
    (void)n;
    int64_t cnt = 0, f = 0;
    for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
        int64_t k = rowidx[p];
        double a_kj = val[p];
        for (int64_t q = colptr[k]; q < colptr[k + 1]; ++q) {
            int64_t i = rowidx[q];
            if (!seen[i]) {
                seen[i] = 1;
                acc[i] = 0.0;
                out[cnt++].r = (int32_t)i;
            }
            acc[i] += val[q] * a_kj;
            ++f;
        }
    }
    for (int64_t e = 0; e < cnt; ++e) {
        out[e].v = acc[out[e].r];
        seen[out[e].r] = 0;
    }
    *flops = f;
    return cnt;
}

/* The prune rule on a column already sorted by value descending.
 * Returns m*, the length of the kept prefix; *s_out = column sum. */
static int64_t prune_keep_count(const entry_t* e, int64_t cnt, double theta, int64_t K,
                                double p, int64_t K_rec, double* s_out) {
    double s = 0.0;
    for (int64_t i = 0; i < cnt; ++i) s += e[i].v;
    int64_t t = 0;
    while (t < cnt && e[t].v >= theta) ++t;
    double target = p * s;
    int64_t m_rec = cnt;
    double prefix = 0.0;
    for (int64_t m = 0; m <= cnt; ++m) {
        if (prefix >= target) {
            m_rec = m;
            break;
        }
        if (m < cnt) prefix += e[m].v;
    }
    int64_t keep = t < K ? t : K;
    if (m_rec > keep) keep = m_rec;
    if (keep > K_rec) keep = K_rec;
    if (keep > cnt) keep = cnt;
    if (keep < 0) keep = 0;
    *s_out = s;
    return keep;
}

/* Hadamard power r, then divide by the column sum; returns chaos_j. */
static double inflate_normalize_column(entry_t* e, int64_t m, double r) {
    double U = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        e[i].v = pow(e[i].v, r);
        U += e[i].v;
    }
    double mx = 0.0, sq = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        e[i].v = (U > 0.0) ? e[i].v / U : 0.0;
        if (e[i].v > mx) mx = e[i].v;
        sq += e[i].v * e[i].v;
    }
    double c = mx - sq;
    return c > 0.0 ? c : 0.0;
}

static int pick_threads(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int orc_num_threads(int nthreads) { return pick_threads(nthreads); }

/*
 * One MCL iteration (expansion, prune, optional inflation + normalisation,
 * chaos) for the listed columns of A (n x n, CSC, FP64 values).
 *
 * Per listed column c (column j = cols[c]):
 *   flops[c], bnnz[c] = nnz(B_*j), bsum[c] = sum_i b_ij,
 *   ntop[c] = min(bnnz, topcap) and the first ntop entries of B_*j in
 *            (value desc, row asc) order in top_rows/top_vals[c*topcap ...],
 *   mstar[c] = kept count (<= kcap required, else -1 is returned),
 *   out_rows/out_vals[c*kcap ...] = kept entries sorted by row; their values
 *            are inflated + normalised when do_inflate, else the B values,
 *   chaos[c] (0 when do_inflate is 0).
 * Returns 0, or -1 when some kept count exceeded kcap, -2 on allocation failure.
 */
int orc_expand_cols(int64_t n, const int64_t* colptr, const int32_t* rowidx, const double* val,
                    int64_t ncols, const int32_t* cols, double theta, int64_t K, double p,
                    int64_t K_rec, double r, int do_inflate, int64_t topcap, int64_t kcap,
                    int64_t* flops, int64_t* bnnz, double* bsum, int64_t* ntop,
                    int32_t* top_rows, double* top_vals, int64_t* mstar, int32_t* out_rows,
                    double* out_vals, double* chaos, int nthreads) {
    int status = 0;
    int nt = pick_threads(nthreads);
#pragma omp parallel num_threads(nt)
    {
        double* acc = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        unsigned char* seen = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
        entry_t* col = (entry_t*)malloc(sizeof(entry_t) * (size_t)(n > 0 ? n : 1));
        if (!acc || !seen || !col) {
#pragma omp atomic write
            status = -2;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t c = 0; c < ncols; ++c) {
                int64_t j = cols[c];
                int64_t f = 0;
                int64_t cnt = expand_column(n, colptr, rowidx, val, j, acc, seen, col, &f);
                qsort(col, (size_t)cnt, sizeof(entry_t), cmp_value_desc);
                double s = 0.0;
                int64_t keep = prune_keep_count(col, cnt, theta, K, p, K_rec, &s);
                flops[c] = f;
                bnnz[c] = cnt;
                bsum[c] = s;
                int64_t nt_ = cnt < topcap ? cnt : topcap;
                ntop[c] = nt_;
                for (int64_t e = 0; e < nt_; ++e) {
                    top_rows[c * topcap + e] = col[e].r;
                    top_vals[c * topcap + e] = col[e].v;
                }
                double ch = 0.0;
                if (do_inflate) ch = inflate_normalize_column(col, keep, r);
                chaos[c] = ch;
                mstar[c] = keep;
                if (keep > kcap) {
#pragma omp atomic write
                    status = -1;
                } else {
                    qsort(col, (size_t)keep, sizeof(entry_t), cmp_row_asc);
                    for (int64_t e = 0; e < keep; ++e) {
                        out_rows[c * kcap + e] = col[e].r;
                        out_vals[c * kcap + e] = col[e].v;
                    }
                }
            }
        }
        free(acc);
        free(seen);
        free(col);
    }
    return status;
}

/*
 * The prune rule alone on the listed columns of a given matrix B (m x ncol
 * CSC, FP64): kept entries sorted by row with their unchanged B values.
 * bsum[c] = column sum, mstar[c] = kept count (<= kcap or -1 is returned).
 */
int orc_prune_cols(const int64_t* colptr, const int32_t* rowidx, const double* val,
                   int64_t ncols, const int32_t* cols, double theta, int64_t K, double p,
                   int64_t K_rec, int64_t kcap, double* bsum, int64_t* mstar,
                   int32_t* out_rows, double* out_vals) {
    int status = 0;
    for (int64_t c = 0; c < ncols; ++c) {
        int64_t j = cols[c];
        int64_t cnt = colptr[j + 1] - colptr[j];
        entry_t* col = (entry_t*)malloc(sizeof(entry_t) * (size_t)(cnt > 0 ? cnt : 1));
        if (!col) return -2;
        for (int64_t e = 0; e < cnt; ++e) {
            col[e].r = rowidx[colptr[j] + e];
            col[e].v = val[colptr[j] + e];
        }
        qsort(col, (size_t)cnt, sizeof(entry_t), cmp_value_desc);
        double s = 0.0;
        int64_t keep = prune_keep_count(col, cnt, theta, K, p, K_rec, &s);
        bsum[c] = s;
        mstar[c] = keep;
        if (keep > kcap) {
            status = -1;
        } else {
            qsort(col, (size_t)keep, sizeof(entry_t), cmp_row_asc);
            for (int64_t e = 0; e < keep; ++e) {
                out_rows[c * kcap + e] = col[e].r;
                out_vals[c * kcap + e] = col[e].v;
            }
        }
        free(col);
    }
    return status;
}

/* Inflation + renormalisation of every column of a CSC, in place; chaos per column. */
void orc_inflate_normalize(int64_t ncol, const int64_t* colptr, double* val, double r,
                           double* chaos) {
    for (int64_t j = 0; j < ncol; ++j) {
        int64_t m = colptr[j + 1] - colptr[j];
        double U = 0.0;
        for (int64_t e = 0; e < m; ++e) {
            val[colptr[j] + e] = pow(val[colptr[j] + e], r);
            U += val[colptr[j] + e];
        }
        double mx = 0.0, sq = 0.0;
        for (int64_t e = 0; e < m; ++e) {
            double a = (U > 0.0) ? val[colptr[j] + e] / U : 0.0;
            val[colptr[j] + e] = a;
            if (a > mx) mx = a;
            sq += a * a;
        }
        double c = mx - sq;
        chaos[j] = c > 0.0 ? c : 0.0;
    }
}

/* chaos_j = max(0, max_i a_ij - sum_i a_ij^2) for every column of a CSC. */
void orc_chaos(int64_t ncol, const int64_t* colptr, const double* val, double* chaos) {
    for (int64_t j = 0; j < ncol; ++j) {
        double mx = 0.0, sq = 0.0;
        for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
            if (val[e] > mx) mx = val[e];
            sq += val[e] * val[e];
        }
        double c = mx - sq;
        chaos[j] = c > 0.0 ? c : 0.0;
    }
}

/* flops_j and nnz(B_*j) (the exact output size) for the listed columns. */
int orc_symbolic_cols(int64_t n, const int64_t* colptr, const int32_t* rowidx, int64_t ncols,
                      const int32_t* cols, int64_t* flops, int64_t* bnnz, int nthreads) {
    int status = 0;
    int nt = pick_threads(nthreads);
#pragma omp parallel num_threads(nt)
    {
        unsigned char* seen = (unsigned char*)calloc((size_t)(n > 0 ? n : 1), 1);
        int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        if (!seen || !list) {
#pragma omp atomic write
            status = -2;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (int64_t c = 0; c < ncols; ++c) {
                int64_t j = cols[c];
                int64_t cnt = 0, f = 0;
                for (int64_t p = colptr[j]; p < colptr[j + 1]; ++p) {
                    int64_t k = rowidx[p];
                    for (int64_t q = colptr[k]; q < colptr[k + 1]; ++q) {
                        int32_t i = rowidx[q];
                        if (!seen[i]) {
                            seen[i] = 1;
                            list[cnt++] = i;
                        }
                        ++f;
                    }
                }
                for (int64_t e = 0; e < cnt; ++e) seen[list[e]] = 0;
                flops[c] = f;
                bnnz[c] = cnt;
            }
        }
        free(seen);
        free(list);
    }
    return status;
}

/* Union-find root with path halving. */
static int64_t uf_find(int64_t* parent, int64_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

/* Connected components of the undirected pattern (entry (i, j) links i and
 * j); labels[v] = smallest vertex id in v's component. */
void orc_components(int64_t n, const int64_t* colptr, const int32_t* rowidx, int32_t* labels) {
    int64_t* parent = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t v = 0; v < n; ++v) parent[v] = v;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t e = colptr[j]; e < colptr[j + 1]; ++e) {
            int64_t a = uf_find(parent, j), b = uf_find(parent, rowidx[e]);
            if (a == b) continue;
            if (a < b) parent[b] = a; else parent[a] = b;  /* smaller id becomes root */
        }
    }
    for (int64_t v = 0; v < n; ++v) labels[v] = (int32_t)uf_find(parent, v);
    free(parent);
}
