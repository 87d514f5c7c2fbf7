/*
 * Geodesic Sinkhorn oracle, C core.  TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, FP64 CPU code for the two loops of the oracle that are too slow in Python:
 * the brute-force nearest-neighbour search that builds the common graph (Sec. 4, first
 * paragraph: "construct a common graph using an affinity kernel") and the Chebyshev heat
 * filter p_K(L, t) applied through the three-term recurrence (Sec. 3.5).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference leg load this
 * file's library.  It shares no code, header, table or helper with the CUDA library.
 * OpenMP is used only to spread independent rows over host cores; every row is computed in
 * the same order as the sequential definition.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Lexicographic order on (squared distance, index): the tie rule of the oracle's kNN. */
static int pair_less(double da, int64_t ia, double db, int64_t ib)
{
    return (da < db) || (da == db && ia < ib);
}

/*
 * k nearest neighbours of the points rows[0..nr) among all n points of X (row-major [n, d]).
 *
 * Squared distance by direct differences, sum_c (x_q,c - x_j,c)^2 in FP64, the point itself
 * excluded, order by (squared distance, index).  Outputs idx[nr, k] and dist[nr, k] (the
 * Euclidean distance, sqrt of the squared one).  Returns 0, or -1 on bad arguments.
 */
int or_knn_rows(const double *X, int64_t n, int d, int k, const int64_t *rows, int64_t nr,
                int32_t *idx, double *dist)
{
    if (n < 2 || d < 1 || k < 1 || k >= n) return -1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nr; ++r) {
        int64_t q = rows[r];
        if (q < 0 || q >= n) { bad = 1; continue; }
        double *bd = (double *)malloc(sizeof(double) * (size_t)k);
        int64_t *bj = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
        int filled = 0;
        const double *xq = X + q * d;
        for (int64_t j = 0; j < n; ++j) {
            if (j == q) continue;
            const double *xj = X + j * d;
            double s = 0.0;
            for (int c = 0; c < d; ++c) {
                double diff = xq[c] - xj[c];
                s += diff * diff;
            }
            if (filled == k && !pair_less(s, j, bd[k - 1], bj[k - 1])) continue;
            /* insertion into the sorted list of the best candidates so far */
            int p = (filled < k) ? filled : k - 1;
            while (p > 0 && pair_less(s, j, bd[p - 1], bj[p - 1])) {
                bd[p] = bd[p - 1];
                bj[p] = bj[p - 1];
                --p;
            }
            bd[p] = s;
            bj[p] = j;
            if (filled < k) ++filled;
        }
        for (int c = 0; c < k; ++c) {
            idx[r * k + c] = (int32_t)bj[c];
            dist[r * k + c] = sqrt(bd[c]);
        }
        free(bd);
        free(bj);
    }
    return bad ? -1 : 0;
}

/* Y[n, B] = M X for a CSR matrix M (rowptr int64, col int32, val FP64); row-major blocks. */
static void csr_mm(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                   int B, const double *X, double *Y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double *yi = Y + i * B;
        for (int c = 0; c < B; ++c) yi[c] = 0.0;
        for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
            const double m = val[e];
            const double *xj = X + (int64_t)col[e] * B;
            for (int c = 0; c < B; ++c) yi[c] += m * xj[c];
        }
    }
}

/*
 * Chebyshev heat filter (Sec. 3.5): Y = p_K(L, t) V = (b_0 / 2) V + sum_{k=1..K} b_k T_k(Ls) V,
 * with Ls = L - Id the shifted Laplacian given in CSR form and the coefficients b[0..K] as the
 * paper writes them (b_0 is halved here, as in the printed expansion).  T_0(y) = 1 (the
 * standard first polynomial), T_1(y) = y, T_k(y) = 2 y T_{k-1}(y) - T_{k-2}(y).
 * V and Y are row-major [n, B] FP64.  Returns 0, or -1 on bad arguments.
 */
int or_cheb_filter(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                   int K, const double *b, int B, const double *V, double *Y)
{
    if (n < 1 || K < 1 || B < 1) return -1;
    const size_t sz = sizeof(double) * (size_t)n * (size_t)B;
    double *t_prev = (double *)malloc(sz);  /* T_{k-2} V */
    double *t_cur = (double *)malloc(sz);   /* T_{k-1} V */
    double *t_next = (double *)malloc(sz);  /* T_k V */
    double *tmp = (double *)malloc(sz);
    if (!t_prev || !t_cur || !t_next || !tmp) {
        free(t_prev); free(t_cur); free(t_next); free(tmp);
        return -2;
    }
    const int64_t nb = n * (int64_t)B;
    memcpy(t_prev, V, sz);                           /* T_0 V = V          */
    csr_mm(n, rowptr, col, val, B, V, t_cur);        /* T_1 V = Ls V       */
    for (int64_t e = 0; e < nb; ++e) Y[e] = 0.5 * b[0] * t_prev[e] + b[1] * t_cur[e];
    for (int k = 2; k <= K; ++k) {
        csr_mm(n, rowptr, col, val, B, t_cur, tmp);  /* Ls T_{k-1} V       */
        for (int64_t e = 0; e < nb; ++e) {
            t_next[e] = 2.0 * tmp[e] - t_prev[e];
            Y[e] += b[k] * t_next[e];
        }
        double *r = t_prev;
        t_prev = t_cur;
        t_cur = t_next;
        t_next = r;
    }
    free(t_prev); free(t_cur); free(t_next); free(tmp);
    return 0;
}
