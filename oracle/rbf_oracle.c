/*
 * Plain FP64 CPU oracle for Gaussian-RBF implicit surface reconstruction
 * (Cuomo, Galletti, Giunta, Starace, "Surface Reconstruction from Scattered
 * Point via RBF Interpolation on GPU").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path links or calls this
 * file; only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, constant or helper with the CUDA
 * implementation.
 *
 * Every routine is the plain definition written out in double precision:
 *   - off-surface centres x_{N+i} = x_i + delta n_i, x_{2N+i} = x_i - delta n_i
 *     (Section II.A.1) with targets 0 / +t / -t (Section II.A.2);
 *   - Gaussian entries A_ij = exp(-|x_i - x_j|^2 / (2 sigma^2)) (Eq.
 *     matrixEntries, the 1/(sqrt(2 pi) sigma) prefactor dropped: it rescales the
 *     weights only and leaves P_f unchanged), optionally truncated to zero for
 *     |x_i - x_j| >= k sigma (Section III.A, "finite bandwidth");
 *   - the interpolation system A c = b (Eq. RBFsys) solved by an unpivoted
 *     right-looking Cholesky factorisation A = L L^T (A is symmetric positive
 *     definite, Section II.B);
 *   - evaluation P_f(xi) = sum_j c_j phi(|xi - x_j|) (Eq. matxvet).
 * Row sums are accumulated in index order j = 0..n-1 (or cell by cell when a
 * cell list only skips pairs that are provably beyond the cut-off).  OpenMP
 * only splits independent rows between threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Section II.A.1 / II.A.2: the extended data set X u X+ u X- and its targets.
 * C is (3N x 3) row-major, b is 3N.  Targets: 0 on X, +tval on X+, -tval on X-. */
void or_build_centers(const float *pts, const float *nrm, int64_t N, double delta,
                      double tval, double *C, double *b) {
    for (int64_t i = 0; i < N; ++i) {
        for (int d = 0; d < 3; ++d) {
            double x = (double)pts[3 * i + d], nn = (double)nrm[3 * i + d];
            C[3 * i + d] = x;
            C[3 * (N + i) + d] = x + delta * nn;
            C[3 * (2 * N + i) + d] = x - delta * nn;
        }
        b[i] = 0.0;
        b[N + i] = tval;
        b[2 * N + i] = -tval;
    }
}

static inline double sqdist(const double *a, const double *b) {
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return dx * dx + dy * dy + dz * dz;
}

/* Gaussian kernel value for squared distance r2; rc2 <= 0 means no cut-off. */
static inline double phi(double r2, double inv2s2, double rc2) {
    if (rc2 > 0.0 && !(r2 < rc2)) return 0.0;
    return exp(-r2 * inv2s2);
}

/* Eq. RBFsys / matrixEntries: dense n x n matrix, row-major. */
void or_dense_matrix(const double *C, int64_t n, double sigma, double k, double *A) {
    double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    double rc2 = k > 0.0 ? (k * sigma) * (k * sigma) : 0.0;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            A[i * n + j] = phi(sqdist(C + 3 * i, C + 3 * j), inv2s2, rc2);
}

/* Unpivoted right-looking Cholesky, in place on the lower triangle of the
 * row-major n x n matrix A (the strict upper triangle is zeroed on exit).
 * Returns 0 on success or j+1 when the j-th pivot is not positive. */
int or_cholesky(double *A, int64_t n) {
    for (int64_t j = 0; j < n; ++j) {
        double d = A[j * n + j];
        if (!(d > 0.0)) return (int)(j + 1);
        double l = sqrt(d);
        A[j * n + j] = l;
        for (int64_t i = j + 1; i < n; ++i) A[i * n + j] /= l;
        /* trailing update A[i][c] -= L[i][j] L[c][j] for j < c <= i */
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = j + 1; i < n; ++i) {
            double lij = A[i * n + j];
            for (int64_t c = j + 1; c <= i; ++c) A[i * n + c] -= lij * A[c * n + j];
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t c = i + 1; c < n; ++c) A[i * n + c] = 0.0;
    return 0;
}

/* Solve L L^T x = b given the factor from or_cholesky. */
void or_chol_solve(const double *L, int64_t n, const double *b, double *x) {
    for (int64_t i = 0; i < n; ++i) {
        double s = b[i];
        for (int64_t c = 0; c < i; ++c) s -= L[i * n + c] * x[c];
        x[i] = s / L[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (int64_t r = i + 1; r < n; ++r) s -= L[r * n + i] * x[r];
        x[i] = s / L[i * n + i];
    }
}

/* ---- a plain uniform-grid bucket list of the centres (cell edge = cut-off) ---- */
typedef struct {
    double lo[3], h;
    int64_t dim[3];
    int64_t *start; /* ncell + 1 */
    int64_t *idx;   /* n */
} bucket_t;

static int bucket_build(bucket_t *B, const double *C, int64_t n, double h) {
    for (int d = 0; d < 3; ++d) B->lo[d] = INFINITY;
    double hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            if (C[3 * i + d] < B->lo[d]) B->lo[d] = C[3 * i + d];
            if (C[3 * i + d] > hi[d]) hi[d] = C[3 * i + d];
        }
    B->h = h;
    int64_t ncell = 1;
    for (int d = 0; d < 3; ++d) {
        B->dim[d] = (int64_t)floor((hi[d] - B->lo[d]) / h) + 1;
        ncell *= B->dim[d];
    }
    B->start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    B->idx = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *cell = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!B->start || !B->idx || !cell) { free(cell); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        int64_t q[3];
        for (int d = 0; d < 3; ++d) {
            q[d] = (int64_t)floor((C[3 * i + d] - B->lo[d]) / h);
            if (q[d] < 0) q[d] = 0;
            if (q[d] >= B->dim[d]) q[d] = B->dim[d] - 1;
        }
        cell[i] = q[0] + B->dim[0] * (q[1] + B->dim[1] * q[2]);
        B->start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) B->start[c + 1] += B->start[c];
    int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    if (!fill) { free(cell); return -1; }
    memcpy(fill, B->start, (size_t)ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) B->idx[fill[cell[i]]++] = i;
    free(fill);
    free(cell);
    return 0;
}

static void bucket_free(bucket_t *B) {
    free(B->start);
    free(B->idx);
}

/* Sum over centres j with |p - x_j| < rc of w_j exp(-|p - x_j|^2/(2 sigma^2)),
 * using the bucket list to skip cells that lie entirely beyond the cut-off. */
static double kernel_sum_point(const bucket_t *B, const double *C, const double *w,
                               const double *p, double inv2s2, double rc2,
                               int64_t *npairs) {
    int64_t q[3];
    for (int d = 0; d < 3; ++d) q[d] = (int64_t)floor((p[d] - B->lo[d]) / B->h);
    double s = 0.0;
    int64_t cnt = 0;
    for (int64_t cz = q[2] - 1; cz <= q[2] + 1; ++cz) {
        if (cz < 0 || cz >= B->dim[2]) continue;
        for (int64_t cy = q[1] - 1; cy <= q[1] + 1; ++cy) {
            if (cy < 0 || cy >= B->dim[1]) continue;
            for (int64_t cx = q[0] - 1; cx <= q[0] + 1; ++cx) {
                if (cx < 0 || cx >= B->dim[0]) continue;
                int64_t c = cx + B->dim[0] * (cy + B->dim[1] * cz);
                for (int64_t t = B->start[c]; t < B->start[c + 1]; ++t) {
                    int64_t j = B->idx[t];
                    double r2 = sqdist(p, C + 3 * j);
                    if (r2 < rc2) {
                        s += w[j] * exp(-r2 * inv2s2);
                        ++cnt;
                    }
                }
            }
        }
    }
    if (npairs) *npairs += cnt;
    return s;
}

/* y[r] = sum_j Atilde[rows[r], j] z_j for the requested rows (Section III.A:
 * truncated Gaussian, cut-off k sigma, k <= 0 meaning untruncated).  Also
 * returns the number of (i, j) pairs with |x_i - x_j| < k sigma, i = j included,
 * summed over the requested rows.  Returns 0, or -1 on allocation failure. */
int or_kernel_rows(const double *C, int64_t n, double sigma, double k, const double *z,
                   const int64_t *rows, int64_t nrows, double *y, int64_t *pair_count) {
    double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    int64_t total = 0;
    if (k <= 0.0) {
#pragma omp parallel for schedule(static) reduction(+ : total)
        for (int64_t r = 0; r < nrows; ++r) {
            const double *p = C + 3 * rows[r];
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s += z[j] * exp(-sqdist(p, C + 3 * j) * inv2s2);
            y[r] = s;
            total += n;
        }
        if (pair_count) *pair_count = total;
        return 0;
    }
    double rc = k * sigma, rc2 = rc * rc;
    bucket_t B;
    if (bucket_build(&B, C, n, rc) != 0) { bucket_free(&B); return -1; }
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t cnt = 0;
        y[r] = kernel_sum_point(&B, C, z, C + 3 * rows[r], inv2s2, rc2, &cnt);
        total += cnt;
    }
    bucket_free(&B);
    if (pair_count) *pair_count = total;
    return 0;
}

/* Eq. matxvet: f(p_m) = sum_j w_j phi(|p_m - x_j|) at m arbitrary points P
 * (m x 3), truncated at k sigma when k > 0. */
int or_eval_points(const double *C, int64_t n, const double *w, double sigma, double k,
                   const double *P, int64_t m, double *f) {
    double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    if (k <= 0.0) {
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < m; ++r) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s += w[j] * exp(-sqdist(P + 3 * r, C + 3 * j) * inv2s2);
            f[r] = s;
        }
        return 0;
    }
    double rc = k * sigma, rc2 = rc * rc;
    bucket_t B;
    if (bucket_build(&B, C, n, rc) != 0) { bucket_free(&B); return -1; }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < m; ++r) {
        const double *p = P + 3 * r;
        int64_t q[3], inside = 1;
        for (int d = 0; d < 3; ++d) {
            q[d] = (int64_t)floor((p[d] - B.lo[d]) / B.h);
            if (q[d] < -1 || q[d] > B.dim[d]) inside = 0;
        }
        f[r] = inside ? kernel_sum_point(&B, C, w, p, inv2s2, rc2, NULL) : 0.0;
    }
    bucket_free(&B);
    return 0;
}
