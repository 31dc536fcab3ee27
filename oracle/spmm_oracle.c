/*
 * FP64 CPU oracle for CSR SpMM and the operations around it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link,
 * load or call this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Every routine is the plain definition of what it computes, written as loops
 * in the order a reader would check against the paper, in double precision.
 * Rows are distributed over OpenMP threads where a routine is parallel, but the
 * order of additions inside one output element is always the sequential one,
 * so results do not depend on the thread count.
 *
 * Notation follows the paper (Section 1, Section 2.2): A is m x k in CSR form
 * (row offsets row_ptr[m+1], column indices col_ind[nnz], values val[nnz]),
 * B is k x n row-major with leading dimension ldb, C = A B is m x n row-major.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/*
 * C = A B (Section 1 problem statement; Algorithm 1 output "C <- AB").
 * C[i][j] = sum over p in [row_ptr[i], row_ptr[i+1]) of val[p] * B[col_ind[p]][j].
 * Empty rows give zero rows.  Duplicated column indices are summed.
 */
void oracle_spmm_f64(int64_t m, int64_t n, const int32_t *row_ptr, const int32_t *col_ind,
                     const double *val, const double *B, int64_t ldb, double *C, int64_t ldc) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i) {
        double *c = C + i * ldc;
        for (int64_t j = 0; j < n; ++j) c[j] = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            const double a = val[p];
            const double *b = B + (int64_t)col_ind[p] * ldb;
            for (int64_t j = 0; j < n; ++j) c[j] += a * b[j];
        }
    }
}

/*
 * The same product restricted to the listed rows: out[t][j] = C[rows[t]][j].
 * Used to check a sample of a large result one row at a time.
 */
void oracle_spmm_rows_f64(int64_t nrows, const int64_t *rows, int64_t n, const int32_t *row_ptr,
                          const int32_t *col_ind, const double *val, const double *B, int64_t ldb,
                          double *out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nrows; ++t) {
        const int64_t i = rows[t];
        double *c = out + t * n;
        for (int64_t j = 0; j < n; ++j) c[j] = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            const double a = val[p];
            const double *b = B + (int64_t)col_ind[p] * ldb;
            for (int64_t j = 0; j < n; ++j) c[j] += a * b[j];
        }
    }
}

/*
 * Error scale of the acceptance metric: D = |A| |B| (elementwise absolute values),
 * D[i][j] = sum_p |val[p]| * |B[col_ind[p]][j]|, for the listed rows.
 */
void oracle_absbound_rows_f64(int64_t nrows, const int64_t *rows, int64_t n, const int32_t *row_ptr,
                              const int32_t *col_ind, const double *val, const double *B, int64_t ldb,
                              double *out) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nrows; ++t) {
        const int64_t i = rows[t];
        double *c = out + t * n;
        for (int64_t j = 0; j < n; ++j) c[j] = 0.0;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            const double a = fabs(val[p]);
            const double *b = B + (int64_t)col_ind[p] * ldb;
            for (int64_t j = 0; j < n; ++j) c[j] += a * fabs(b[j]);
        }
    }
}

/*
 * Transposed product dB = A^T dC (the SpMM_T operation named in Section 6),
 * written directly from the definition dB[c][j] = sum over (i, p) with
 * col_ind[p] = c of val[p] * dC[i][j], without forming A^T.
 * Threads split the column range j, so every dB element is summed in the
 * sequential (i, p) order.
 */
void oracle_spmm_t_f64(int64_t m, int64_t k, int64_t n, const int32_t *row_ptr, const int32_t *col_ind,
                       const double *val, const double *dC, int64_t lddc, double *dB, int64_t lddb) {
    for (int64_t c = 0; c < k; ++c)
        for (int64_t j = 0; j < n; ++j) dB[c * lddb + j] = 0.0;
#pragma omp parallel
    {
        int64_t nt = 1, me = 0;
#ifdef _OPENMP
        nt = omp_get_num_threads();
        me = omp_get_thread_num();
#endif
        const int64_t j0 = n * me / nt, j1 = n * (me + 1) / nt;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
                const double a = val[p];
                double *d = dB + (int64_t)col_ind[p] * lddb;
                const double *g = dC + i * lddc;
                for (int64_t j = j0; j < j1; ++j) d[j] += a * g[j];
            }
    }
}

/*
 * Sampled dense-dense product on A's pattern (the gradient of <G, A B> with
 * respect to the stored values): out[p] = sum_j dC[i][j] * B[col_ind[p]][j]
 * for every nonzero p of row i.
 */
void oracle_sddmm_f64(int64_t m, int64_t n, const int32_t *row_ptr, const int32_t *col_ind,
                      const double *dC, int64_t lddc, const double *B, int64_t ldb, double *out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            const double *g = dC + i * lddc;
            const double *b = B + (int64_t)col_ind[p] * ldb;
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s += g[j] * b[j];
            out[p] = s;
        }
}

/*
 * |dC| |B|^T on the pattern: the error scale of the SDDMM result,
 * out[p] = sum_j |dC[i][j]| * |B[col_ind[p]][j]|.
 */
void oracle_sddmm_absbound_f64(int64_t m, int64_t n, const int32_t *row_ptr, const int32_t *col_ind,
                               const double *dC, int64_t lddc, const double *B, int64_t ldb, double *out) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            const double *g = dC + i * lddc;
            const double *b = B + (int64_t)col_ind[p] * ldb;
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s += fabs(g[j]) * fabs(b[j]);
            out[p] = s;
        }
}

/*
 * CSR transpose by a stable counting sort on the column index.
 * Row c of A^T lists, in increasing original position p, every nonzero p of A
 * with col_ind[p] = c: col_ind_t holds its row i, perm holds p, so that
 * val_t[q] = val[perm[q]].  row_ptr_t has k + 1 entries.
 */
void oracle_csr_transpose(int64_t m, int64_t k, const int32_t *row_ptr, const int32_t *col_ind,
                          int32_t *row_ptr_t, int32_t *col_ind_t, int32_t *perm) {
    const int64_t nnz = m > 0 ? row_ptr[m] : 0;
    int64_t *next = (int64_t *)calloc((size_t)(k + 1), sizeof(int64_t));
    for (int64_t p = 0; p < nnz; ++p) next[col_ind[p] + 1] += 1;
    for (int64_t c = 0; c < k; ++c) next[c + 1] += next[c];
    for (int64_t c = 0; c <= k; ++c) row_ptr_t[c] = (int32_t)next[c];
    for (int64_t i = 0; i < m; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            const int64_t q = next[col_ind[p]]++;
            col_ind_t[q] = (int32_t)i;
            perm[q] = (int32_t)p;
        }
    free(next);
}

/*
 * Merge-path decomposition (Section 4, item 2(b); Fig. 2(c)), by its definition:
 * merge the list of row end offsets row_ptr[1..m] with the list of nonzero
 * indices 0..nnz-1, taking a row end first when it is <= the next nonzero index.
 * Walking the merged sequence, limits[2t], limits[2t+1] record (rows consumed,
 * nonzeros consumed) after min(t * items, m + nnz) steps, for t = 0..tiles.
 */
void oracle_merge_path_limits(int64_t m, const int32_t *row_ptr, int64_t items, int64_t tiles,
                              int32_t *limits) {
    const int64_t nnz = m > 0 ? row_ptr[m] : 0;
    const int64_t total = m + nnz;
    int64_t r = 0, z = 0, step = 0;
    for (int64_t t = 0; t <= tiles; ++t) {
        int64_t target = t * items;
        if (target > total) target = total;
        while (step < target) {
            if (r < m && row_ptr[r + 1] <= z) ++r;
            else ++z;
            ++step;
        }
        limits[2 * t] = (int32_t)r;
        limits[2 * t + 1] = (int32_t)z;
    }
}

/*
 * SpMM over a semiring (the GraphBLAS matrix-matrix product named in
 * Section 1): C[i][j] = (+) over p in row i of (val[p] (x) B[col_ind[p]][j]),
 * starting from the identity of (+); an empty row gives the identity.
 * semiring 0: (+, x) with identity 0; 1: (min, +) with identity +inf;
 * 2: (max, +) with identity -inf; 3: (max, x) with identity -inf.
 */
void oracle_spmm_semiring_f64(int64_t m, int64_t n, int semiring, const int32_t *row_ptr, const int32_t *col_ind,
                              const double *val, const double *B, int64_t ldb, double *C, int64_t ldc) {
    const double ident = semiring == 0 ? 0.0 : semiring == 1 ? INFINITY : -INFINITY;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < m; ++i) {
        double *c = C + i * ldc;
        for (int64_t j = 0; j < n; ++j) c[j] = ident;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            const double a = val[p];
            const double *b = B + (int64_t)col_ind[p] * ldb;
            for (int64_t j = 0; j < n; ++j) {
                if (semiring == 0) c[j] += a * b[j];
                else if (semiring == 1) c[j] = fmin(c[j], a + b[j]);
                else if (semiring == 2) c[j] = fmax(c[j], a + b[j]);
                else c[j] = fmax(c[j], a * b[j]);
            }
        }
    }
}
