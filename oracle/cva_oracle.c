/*
 * cva_oracle.c -- plain FP64 CPU Canonical Variates Analysis (CVA).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file's library; the CUDA library never does and
 * shares no code with it.  It is written for a reader checking it against the
 * paper by eye: scalar loops, no blocking, no fusion, no reordering.
 *
 * What it computes, in the paper's order (arXiv 1612.06457):
 *   1. counts and sums of the labelled training pixels of each class
 *      (Section 2: points picked per class, a bands x points matrix);
 *   2. class means, the within-class and the between-class scatter
 *      (Section 2: "covariance matrixes within each class and between the
 *      classes"), accumulated in two passes over the training pixels;
 *   3. the eigenanalysis of those two matrices: the generalized
 *      symmetric-definite problem  Sb v = lambda Sw v  (Section 4 solves it
 *      with GSL's generalized symmetric-definite solver), here by the
 *      textbook Cholesky reduction to a standard symmetric problem followed
 *      by the cyclic Jacobi method (Golub and Van Loan, "Matrix
 *      Computations", the symmetric-definite reduction and cyclic Jacobi);
 *   4. the projection of every pixel on the canonical vectors (Section 2:
 *      the coefficients are multiplied with the band images);
 *   5. the linear rescale of each projection to 0..255 (Section 2), with
 *      the range taken either from all pixels or from the training pixels.
 *
 * Readings where the paper is silent (each is also a pinned test):
 *   - Sw and Sb are unnormalised sums of squares and cross-products:
 *       Sw = sum_c sum_{p in c} (x_p - mu_c)(x_p - mu_c)^T
 *       Sb = sum_c n_c (mu_c - mu)(mu_c - mu)^T,   mu = sum_c n_c mu_c / N.
 *     A common rescaling changes lambda by a constant and V by a scalar,
 *     which the 8-bit rescale removes.
 *   - eigenvectors are scaled so that V^T Sw V = I;
 *   - eigenvalues are sorted in descending order;
 *   - the sign of each eigenvector makes its largest-magnitude component
 *     positive; components within 1e-12 (relative) of the largest count as
 *     ties and the lowest band index wins (Section 4 notes that two solvers
 *     return opposite signs);
 *   - projections are centred on the training mean: y_j = v_j^T (x - mu);
 *   - the 8-bit value is floor(255 (y - lo) / (hi - lo) + 1/2) clamped to
 *     0..255, and 0 everywhere when hi <= lo; the 16-bit value (Section 2's
 *     CVA-GSL tool writes 8- and 16-bit images) the same with 65535;
 *   - principal components (Section 2: the unsupervised PCA of the whole
 *     page, optionally cropped to the folio) are the eigenvectors of the
 *     sample covariance sum_p (x_p - mu)(x_p - mu)^T / (N - 1) of the
 *     selected pixels, orthonormal, with the same order and sign convention;
 *     they come from the same solver with Sw = I;
 *   - the third rescale takes p percent of the pixels out of EACH tail:
 *     with m = floor(p P / 100), lo is the (m+1)-th smallest and hi the
 *     (m+1)-th largest value of the projection, p in steps of 0.01 below 50
 *     (the paper's values are 0.01, 0.1, 1 and 5);
 *   - Sw is "not positive definite" when a Cholesky pivot falls to or below
 *     1e-12 times its own diagonal entry of Sw; no ridge is added.
 *
 * Threads: built plainly this file is single-threaded.  Built with
 * -fopenmp (a second library, used only to time the oracle on every host
 * core) the per-pixel loops of the projection, the ranges, the rescales and
 * the integer class sums run over the pixels in parallel; each of those
 * results is independent of the order in which pixels are visited (one
 * value per pixel, exact integer sums, min / max), so both builds give
 * identical results.  The FP64 scatter sums stay serial for that reason.
 *
 * Layouts: cube is band-sequential uint16 B x P (P = H W pixels, band b at
 * cube + b P); labels are uint8 P, 0 = not a training pixel, c + 1 = class c;
 * all matrices are row-major doubles; V column j is canonical vector j; a
 * projection is k x P doubles; a range is 2 k doubles (lo_j, hi_j) pairs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_EMPTY_CLASS (-2)
#define ORC_ERR_NOT_SPD (-3)
#define ORC_ERR_NO_CONVERGENCE (-4)
#define ORC_ERR_LABEL (-7)

#define ORC_PIVOT_REL 1e-12
#define ORC_TIE_REL 1e-12
#define ORC_MAX_SWEEPS 100

/* ------------------------------------------------------------------------ */
/* 1. training counts and sums (Section 2)                                   */
/* ------------------------------------------------------------------------ */

/* n[c] = number of pixels labelled c + 1; s[c*B + b] = sum of band b over
 * them.  Exact in 64-bit integers.  Returns ORC_ERR_LABEL if a label exceeds K. */
int orc_class_sums(const uint16_t* cube, int64_t B, int64_t P, const uint8_t* labels, int64_t K,
                   int64_t* n, int64_t* s)
{
    if (B < 1 || P < 0 || K < 1) return ORC_ERR_ARG;
    for (int64_t c = 0; c < K; ++c) {
        n[c] = 0;
        for (int64_t b = 0; b < B; ++b) s[c * B + b] = 0;
    }
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : n[:K], s[:K * B]) reduction(| : bad)
    for (int64_t p = 0; p < P; ++p) {
        int64_t lab = labels[p];
        if (lab == 0) continue;
        if (lab > K) { bad = 1; continue; }
        int64_t c = lab - 1;
        n[c] += 1;
        for (int64_t b = 0; b < B; ++b) s[c * B + b] += cube[b * P + p];
    }
    return bad ? ORC_ERR_LABEL : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* 2. means and scatter matrices (Section 2)                                 */
/* ------------------------------------------------------------------------ */

/* mu_c (K x B), mu (B), Sw (B x B), Sb (B x B) from the training pixels.
 * Pass one takes the class means, pass two sums the centred outer products. */
int orc_scatter(const uint16_t* cube, int64_t B, int64_t P, const uint8_t* labels, int64_t K,
                int64_t* n, double* mu_c, double* mu, double* Sw, double* Sb)
{
    int64_t* s = (int64_t*)malloc(sizeof(int64_t) * (size_t)(K * B));
    if (!s) return ORC_ERR_ARG;
    int rc = orc_class_sums(cube, B, P, labels, K, n, s);
    if (rc != ORC_OK) { free(s); return rc; }
    int64_t N = 0;
    for (int64_t c = 0; c < K; ++c) {
        if (n[c] == 0) { free(s); return ORC_ERR_EMPTY_CLASS; }
        N += n[c];
    }
    for (int64_t c = 0; c < K; ++c)
        for (int64_t b = 0; b < B; ++b)
            mu_c[c * B + b] = (double)s[c * B + b] / (double)n[c];
    for (int64_t b = 0; b < B; ++b) {
        int64_t tot = 0;
        for (int64_t c = 0; c < K; ++c) tot += s[c * B + b];
        mu[b] = (double)tot / (double)N;
    }
    free(s);

    for (int64_t i = 0; i < B * B; ++i) { Sw[i] = 0.0; Sb[i] = 0.0; }
    double* d = (double*)malloc(sizeof(double) * (size_t)B);
    if (!d) return ORC_ERR_ARG;
    for (int64_t p = 0; p < P; ++p) {
        int64_t lab = labels[p];
        if (lab == 0) continue;
        int64_t c = lab - 1;
        for (int64_t b = 0; b < B; ++b) d[b] = (double)cube[b * P + p] - mu_c[c * B + b];
        for (int64_t i = 0; i < B; ++i)
            for (int64_t j = 0; j < B; ++j) Sw[i * B + j] += d[i] * d[j];
    }
    for (int64_t c = 0; c < K; ++c) {
        for (int64_t b = 0; b < B; ++b) d[b] = mu_c[c * B + b] - mu[b];
        for (int64_t i = 0; i < B; ++i)
            for (int64_t j = 0; j < B; ++j) Sb[i * B + j] += (double)n[c] * d[i] * d[j];
    }
    free(d);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* 3. generalized symmetric-definite eigenproblem Sb v = lambda Sw v         */
/* ------------------------------------------------------------------------ */

/* Lower Cholesky factor L of A (B x B), row by row.  Returns ORC_ERR_NOT_SPD
 * when a pivot is not above ORC_PIVOT_REL times its diagonal entry of A. */
static int cholesky_lower(int64_t B, const double* A, double* L)
{
    for (int64_t i = 0; i < B * B; ++i) L[i] = 0.0;
    for (int64_t i = 0; i < B; ++i) {
        for (int64_t j = 0; j <= i; ++j) {
            double sum = A[i * B + j];
            for (int64_t k = 0; k < j; ++k) sum -= L[i * B + k] * L[j * B + k];
            if (i == j) {
                if (!(sum > ORC_PIVOT_REL * A[i * B + i])) return ORC_ERR_NOT_SPD;
                L[i * B + i] = sqrt(sum);
            } else {
                L[i * B + j] = sum / L[j * B + j];
            }
        }
    }
    return ORC_OK;
}

/* Solve L x = r in place (forward substitution); r has stride `inc`. */
static void forward_solve(int64_t B, const double* L, double* r, int64_t inc)
{
    for (int64_t i = 0; i < B; ++i) {
        double sum = r[i * inc];
        for (int64_t k = 0; k < i; ++k) sum -= L[i * B + k] * r[k * inc];
        r[i * inc] = sum / L[i * B + i];
    }
}

/* Solve L^T x = r in place (back substitution); r has stride `inc`. */
static void back_solve_transposed(int64_t B, const double* L, double* r, int64_t inc)
{
    for (int64_t i = B - 1; i >= 0; --i) {
        double sum = r[i * inc];
        for (int64_t k = i + 1; k < B; ++k) sum -= L[k * B + i] * r[k * inc];
        r[i * inc] = sum / L[i * B + i];
    }
}

/* Cyclic Jacobi on the symmetric C (B x B, overwritten): on exit the
 * diagonal of C holds the eigenvalues and U (B x B) the eigenvectors as
 * columns.  Sweeps go row by row over p < q until the off-diagonal norm is
 * below 1e-15 of the Frobenius norm. */
static int jacobi_cyclic(int64_t B, double* C, double* U, int* sweeps_out)
{
    for (int64_t i = 0; i < B; ++i)
        for (int64_t j = 0; j < B; ++j) U[i * B + j] = (i == j) ? 1.0 : 0.0;
    double fro = 0.0;
    for (int64_t i = 0; i < B * B; ++i) fro += C[i] * C[i];
    fro = sqrt(fro);
    int sweep = 0;
    for (;;) {
        double off = 0.0;
        for (int64_t p = 0; p < B; ++p)
            for (int64_t q = 0; q < B; ++q)
                if (p != q) off += C[p * B + q] * C[p * B + q];
        off = sqrt(off);
        if (off <= 1e-15 * fro || off == 0.0) break;
        if (sweep >= ORC_MAX_SWEEPS) { *sweeps_out = sweep; return ORC_ERR_NO_CONVERGENCE; }
        ++sweep;
        for (int64_t p = 0; p < B - 1; ++p) {
            for (int64_t q = p + 1; q < B; ++q) {
                double apq = C[p * B + q];
                if (apq == 0.0) continue;
                /* rotation angle that zeroes C[p][q] */
                double tau = (C[q * B + q] - C[p * B + p]) / (2.0 * apq);
                double t;
                if (fabs(tau) > 1e150) t = 0.5 / tau;
                else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double cs = 1.0 / sqrt(1.0 + t * t);
                double sn = t * cs;
                /* C <- C J : columns p and q */
                for (int64_t r = 0; r < B; ++r) {
                    double a = C[r * B + p], b = C[r * B + q];
                    C[r * B + p] = cs * a - sn * b;
                    C[r * B + q] = sn * a + cs * b;
                }
                /* C <- J^T C : rows p and q */
                for (int64_t r = 0; r < B; ++r) {
                    double a = C[p * B + r], b = C[q * B + r];
                    C[p * B + r] = cs * a - sn * b;
                    C[q * B + r] = sn * a + cs * b;
                }
                /* U <- U J */
                for (int64_t r = 0; r < B; ++r) {
                    double a = U[r * B + p], b = U[r * B + q];
                    U[r * B + p] = cs * a - sn * b;
                    U[r * B + q] = sn * a + cs * b;
                }
            }
        }
    }
    *sweeps_out = sweep;
    return ORC_OK;
}

/* lambda (B) descending and V (B x B, column j = vector j, V^T Sw V = I)
 * with the sign convention above.  `sweeps` (may be NULL) gets the Jacobi
 * sweep count. */
int orc_gen_eig(int64_t B, const double* Sw, const double* Sb, double* lambda, double* V, int* sweeps)
{
    if (B < 1) return ORC_ERR_ARG;
    size_t bytes = sizeof(double) * (size_t)(B * B);
    double* L = (double*)malloc(bytes);
    double* C = (double*)malloc(bytes);
    double* U = (double*)malloc(bytes);
    double* W = (double*)malloc(bytes);
    int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)B);
    int rc = ORC_OK, nsw = 0;
    if (!L || !C || !U || !W || !order) { rc = ORC_ERR_ARG; goto done; }

    rc = cholesky_lower(B, Sw, L);
    if (rc != ORC_OK) goto done;

    /* C = L^-1 Sb L^-T: first X = L^-1 Sb column by column, then
     * C = L^-1 X^T column by column (X^T = Sb L^-T since Sb is symmetric). */
    memcpy(C, Sb, bytes);
    for (int64_t j = 0; j < B; ++j) forward_solve(B, L, C + j, B);      /* C = X */
    for (int64_t i = 0; i < B; ++i)
        for (int64_t j = 0; j < B; ++j) W[i * B + j] = C[j * B + i];      /* W = X^T */
    for (int64_t j = 0; j < B; ++j) forward_solve(B, L, W + j, B);      /* W = L^-1 X^T */
    for (int64_t i = 0; i < B; ++i)
        for (int64_t j = 0; j < B; ++j) C[i * B + j] = 0.5 * (W[i * B + j] + W[j * B + i]);

    rc = jacobi_cyclic(B, C, U, &nsw);
    if (rc != ORC_OK) goto done;

    /* V = L^-T U */
    for (int64_t j = 0; j < B; ++j) back_solve_transposed(B, L, U + j, B);

    /* order by descending eigenvalue (insertion sort, stable) */
    for (int64_t i = 0; i < B; ++i) order[i] = i;
    for (int64_t i = 1; i < B; ++i) {
        int64_t o = order[i];
        int64_t j = i - 1;
        while (j >= 0 && C[order[j] * B + order[j]] < C[o * B + o]) { order[j + 1] = order[j]; --j; }
        order[j + 1] = o;
    }
    for (int64_t j = 0; j < B; ++j) {
        int64_t src = order[j];
        lambda[j] = C[src * B + src];
        for (int64_t b = 0; b < B; ++b) V[b * B + j] = U[b * B + src];
    }

    /* sign: largest-magnitude component positive, ties to the lowest band */
    for (int64_t j = 0; j < B; ++j) {
        double big = 0.0;
        for (int64_t b = 0; b < B; ++b) if (fabs(V[b * B + j]) > big) big = fabs(V[b * B + j]);
        int64_t arg = 0;
        for (int64_t b = 0; b < B; ++b) {
            if (fabs(V[b * B + j]) >= big * (1.0 - ORC_TIE_REL)) { arg = b; break; }
        }
        if (V[arg * B + j] < 0.0)
            for (int64_t b = 0; b < B; ++b) V[b * B + j] = -V[b * B + j];
    }

done:
    if (sweeps) *sweeps = nsw;
    free(L); free(C); free(U); free(W); free(order);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* 4. projection on the canonical vectors (Section 2)                        */
/* ------------------------------------------------------------------------ */

/* y[j * (p1 - p0) + (p - p0)] = sum_b V[b][j] (x_b[p] - mu_b) for j < k and
 * p0 <= p < p1.  V is B x ldv row-major (column j = vector j). */
int orc_project(const uint16_t* cube, int64_t B, int64_t P, int64_t p0, int64_t p1,
                const double* V, int64_t ldv, const double* mu, int64_t k, double* y)
{
    if (B < 1 || k < 0 || k > ldv || p0 < 0 || p1 < p0 || p1 > P) return ORC_ERR_ARG;
    int64_t n = p1 - p0;
    for (int64_t j = 0; j < k; ++j) {
#pragma omp parallel for schedule(static)
        for (int64_t p = p0; p < p1; ++p) {
            double acc = 0.0;
            for (int64_t b = 0; b < B; ++b) acc += V[b * ldv + j] * ((double)cube[b * P + p] - mu[b]);
            y[j * n + (p - p0)] = acc;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* 5. ranges and the 8-bit rescale (Section 2)                               */
/* ------------------------------------------------------------------------ */

/* Range over all P pixels of each of the k projections (first rescale). */
void orc_range_global(const double* y, int64_t k, int64_t P, double* range)
{
    for (int64_t j = 0; j < k; ++j) {
        double lo = INFINITY, hi = -INFINITY;
#pragma omp parallel for schedule(static) reduction(min : lo) reduction(max : hi)
        for (int64_t p = 0; p < P; ++p) {
            double v = y[j * P + p];
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        range[2 * j] = lo;
        range[2 * j + 1] = hi;
    }
}

/* Range over the training pixels only (second rescale: the scores of the
 * input points set the 0..255 end points). */
void orc_range_training(const double* y, int64_t k, int64_t P, const uint8_t* labels, double* range)
{
    for (int64_t j = 0; j < k; ++j) {
        double lo = INFINITY, hi = -INFINITY;
#pragma omp parallel for schedule(static) reduction(min : lo) reduction(max : hi)
        for (int64_t p = 0; p < P; ++p) {
            if (labels[p] == 0) continue;
            double v = y[j * P + p];
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        range[2 * j] = lo;
        range[2 * j + 1] = hi;
    }
}

/* out[j * P + p] = clamp(floor(255 (y - lo) / (hi - lo) + 1/2), 0, 255). */
void orc_to_u8(const double* y, int64_t k, int64_t P, const double* range, uint8_t* out)
{
    for (int64_t j = 0; j < k; ++j) {
        double lo = range[2 * j], hi = range[2 * j + 1];
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < P; ++p) {
            double v = 0.0;
            if (hi > lo) v = floor(255.0 * (y[j * P + p] - lo) / (hi - lo) + 0.5);
            if (v < 0.0) v = 0.0;
            if (v > 255.0) v = 255.0;
            out[j * P + p] = (uint8_t)v;
        }
    }
}


/* out[j * P + p] = clamp(floor(65535 (y - lo) / (hi - lo) + 1/2), 0, 65535). */
void orc_to_u16(const double* y, int64_t k, int64_t P, const double* range, uint16_t* out)
{
    for (int64_t j = 0; j < k; ++j) {
        double lo = range[2 * j], hi = range[2 * j + 1];
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < P; ++p) {
            double v = 0.0;
            if (hi > lo) v = floor(65535.0 * (y[j * P + p] - lo) / (hi - lo) + 0.5);
            if (v < 0.0) v = 0.0;
            if (v > 65535.0) v = 65535.0;
            out[j * P + p] = (uint16_t)v;
        }
    }
}

static int cmp_double(const void* a, const void* b)
{
    const double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* The third rescale's range (Section 2: "taking out" a percentile of the
 * data): with bp = p * 100 (p in percent, steps of 0.01, p < 50) and
 * m = floor(bp P / 10000) values taken out of each tail, lo_j is the
 * (m+1)-th smallest and hi_j the (m+1)-th largest of the P values of
 * projection j.  bp = 0 gives the global range. */
int orc_percentile_range(const double* y, int64_t k, int64_t P, int64_t bp, double* range)
{
    if (k < 1 || P < 1 || bp < 0 || bp > 4999) return ORC_ERR_ARG;
    double* v = (double*)malloc(sizeof(double) * (size_t)P);
    if (!v) return ORC_ERR_ARG;
    const int64_t m = (bp * P) / 10000;
    for (int64_t j = 0; j < k; ++j) {
        memcpy(v, y + j * P, sizeof(double) * (size_t)P);
        qsort(v, (size_t)P, sizeof(double), cmp_double);
        range[2 * j] = v[m];
        range[2 * j + 1] = v[P - 1 - m];
    }
    free(v);
    return ORC_OK;
}


/* Mean and sample covariance of the pixels selected by mask (all pixels when
 * mask is NULL), in two passes: mu = sum x_p / N, then
 * C = sum (x_p - mu)(x_p - mu)^T / (N - 1).  *N_out = N. */
int orc_pca_cov(const uint16_t* cube, int64_t B, int64_t P, const uint8_t* mask, double* mu, double* C,
                int64_t* N_out)
{
    if (B < 1 || P < 1) return ORC_ERR_ARG;
    int64_t N = 0;
    for (int64_t b = 0; b < B; ++b) mu[b] = 0.0;
    for (int64_t p = 0; p < P; ++p) {
        if (mask && mask[p] == 0) continue;
        ++N;
        for (int64_t b = 0; b < B; ++b) mu[b] += (double)cube[b * P + p];
    }
    *N_out = N;
    if (N < 2) return ORC_ERR_EMPTY_CLASS;
    for (int64_t b = 0; b < B; ++b) mu[b] /= (double)N;
    for (int64_t i = 0; i < B * B; ++i) C[i] = 0.0;
    double* d = (double*)malloc(sizeof(double) * (size_t)B);
    if (!d) return ORC_ERR_ARG;
    for (int64_t p = 0; p < P; ++p) {
        if (mask && mask[p] == 0) continue;
        for (int64_t b = 0; b < B; ++b) d[b] = (double)cube[b * P + p] - mu[b];
        for (int64_t i = 0; i < B; ++i)
            for (int64_t j = 0; j < B; ++j) C[i * B + j] += d[i] * d[j];
    }
    free(d);
    for (int64_t i = 0; i < B * B; ++i) C[i] /= (double)(N - 1);
    return ORC_OK;
}


/* Cluster-separation indices of the classes of a label map in a k-band image
 * (Section 3, eqs. 1-5; p = 2): for class c with T_c labelled pixels x,
 *   A_c  = the centroid (mean of x),
 *   S_c  = the mean Euclidean distance of its pixels to A_c          (eq. 1)
 * and for a pair of classes
 *   M_ij = ||A_i - A_j||                                             (eq. 2)
 *   R_ij = (S_i + S_j) / M_ij          (Davies-Bouldin ratio,        eq. 3)
 *   DI_ij = (M_ij - S_i - S_j) / max(S_i, S_j)    (Dunn,             eq. 5)
 * y is k x P (doubles), labels P (0 = none, c + 1 = class c).  M, R and DI are
 * K x K; their diagonals are 0; R is +inf when M_ij = 0 and DI is +inf when
 * both scatters are 0. */
int orc_cluster_indices(const double* y, int64_t k, int64_t P, const uint8_t* labels, int64_t K, int64_t* T,
                        double* A, double* S, double* M, double* R, double* DI)
{
    if (k < 1 || P < 0 || K < 1) return ORC_ERR_ARG;
    for (int64_t c = 0; c < K; ++c) {
        T[c] = 0;
        S[c] = 0.0;
        for (int64_t j = 0; j < k; ++j) A[c * k + j] = 0.0;
    }
    for (int64_t p = 0; p < P; ++p) {
        const int64_t lab = labels[p];
        if (lab == 0) continue;
        if (lab > K) return ORC_ERR_LABEL;
        T[lab - 1] += 1;
        for (int64_t j = 0; j < k; ++j) A[(lab - 1) * k + j] += y[j * P + p];
    }
    for (int64_t c = 0; c < K; ++c) {
        if (T[c] == 0) return ORC_ERR_EMPTY_CLASS;
        for (int64_t j = 0; j < k; ++j) A[c * k + j] /= (double)T[c];
    }
    for (int64_t p = 0; p < P; ++p) {
        const int64_t lab = labels[p];
        if (lab == 0) continue;
        double d2 = 0.0;
        for (int64_t j = 0; j < k; ++j) {
            const double d = y[j * P + p] - A[(lab - 1) * k + j];
            d2 += d * d;
        }
        S[lab - 1] += sqrt(d2);
    }
    for (int64_t c = 0; c < K; ++c) S[c] /= (double)T[c];
    for (int64_t i = 0; i < K; ++i)
        for (int64_t j = 0; j < K; ++j) {
            double d2 = 0.0;
            for (int64_t q = 0; q < k; ++q) {
                const double d = A[i * k + q] - A[j * k + q];
                d2 += d * d;
            }
            const double m = sqrt(d2);
            M[i * K + j] = m;
            if (i == j) {
                R[i * K + j] = 0.0;
                DI[i * K + j] = 0.0;
                continue;
            }
            R[i * K + j] = m > 0.0 ? (S[i] + S[j]) / m : INFINITY;
            const double smax = S[i] > S[j] ? S[i] : S[j];
            DI[i * K + j] = smax > 0.0 ? (m - S[i] - S[j]) / smax : INFINITY;
        }
    return ORC_OK;
}

/* Threads the per-pixel loops use: sets them when n > 0 (OpenMP build only)
 * and returns the number in effect (1 in the plain build). */
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
