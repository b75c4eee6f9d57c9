/*
 * Oracle for the dense LU solve (LINPACK / HPL hot path) -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the bench's CPU-baseline arm load this
 * library.  It is a plain, slow, obviously correct FP64 CPU implementation of
 * what the GPU path computes, and it shares no code with the GPU path.
 *
 * What it computes, and the passage of arxiv 2202.13995 each part follows:
 *   - the problem: solve A x = b with A = L U, then L y = b and U x = y
 *     (section "High Performance Linpack", first paragraph);
 *   - orc_getf2: Gaussian elimination with partial pivoting, unblocked and
 *     right-looking, LAPACK dgetf2 semantics: ipiv is 1-based, the pivot is the
 *     first row of largest |a| in the column, a zero pivot sets info to the
 *     first such column and the elimination continues without scaling.  The
 *     paper uses no pivoting (HPL-AI rules, diagonally dominant A); partial
 *     pivoting is the classical HPL rule and what this solver implements;
 *   - orc_getrf_blocked: the paper's blocked right-looking iteration (section
 *     "Base Implementation", figure "lu_iteration"): factor the current block
 *     column (diagonal "LU" block plus the "left" blocks below it, which with
 *     partial pivoting form one panel), apply its row interchanges to the other
 *     columns, update the "top" blocks with L (a unit-lower triangular solve),
 *     then update the "inner" blocks by a matrix multiplication;
 *   - orc_getf2_nopiv / orc_getrf_nopiv_blocked: the paper's own variant
 *     (HPL-AI rules: diagonally dominant A, no pivoting), unblocked and as the
 *     paper's four-kernel blocked iteration (LU, top, left, inner);
 *   - orc_getrs: y = L^-1 P b, x = U^-1 y (HPL section, first paragraph);
 *   - residual and norms: r = b - A x and the HPL scaled residual
 *     ||r||_inf / (eps (||A||_inf ||x||_inf + ||b||_inf) n); the paper's own
 *     formula in its validation paragraph is garbled (it has no residual in
 *     it); this reading takes the HPL form with the unit roundoff eps = 2^-53,
 *     plus the paper-shaped variant ||r||_inf / (n ||b||_inf eps);
 *   - orc_cond1_est: Hager's 1-norm estimate of ||A^-1||_1 with Higham's
 *     refinements (N. J. Higham, ACM TOMS 14(4), 1988, Algorithm 4.1), used to
 *     state how far two backward-stable solves may differ;
 *   - orc_round_bf16 / orc_round_fp16: round-to-nearest-even of an FP32 value
 *     to bfloat16 / IEEE binary16, from the formats' definitions;
 *   - orc_gemm_update: C - A B in FP64, the inner-block update.
 *   - orc_gemm_update_dot2: the same update as accurately as if computed in
 *     twice the working precision and rounded once (the Dot2 algorithm of
 *     T. Ogita, S. M. Rump, S. Oishi, "Accurate sum and dot product", SIAM J.
 *     Sci. Comput. 26, 2005): the reference for an update whose own error is of
 *     the order of FP64 rounding (the error-free-splitting update).
 *
 * Matrices are column-major with a leading dimension; sizes are int64 inside.
 * Compiled with -ffp-contract=off so that x86 and Arm builds round the same way.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, ld) ((int64_t)(i) + (int64_t)(j) * (int64_t)(ld))

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Gaussian elimination with partial pivoting on an m x n block (m >= n or not),
 * unblocked, right-looking.  ipiv[j] (1-based, relative to the block) is the row
 * swapped with row j.  Returns info: 0, or the first j+1 with a zero pivot. */
int orc_getf2(int m, int n, double *A, int lda, int *ipiv) {
    int info = 0;
    int kmax = m < n ? m : n;
    for (int j = 0; j < kmax; ++j) {
        /* pivot search: first index of the largest |a_ij|, i >= j */
        int p = j;
        double best = fabs(A[IDX(j, j, lda)]);
        for (int i = j + 1; i < m; ++i) {
            double v = fabs(A[IDX(i, j, lda)]);
            if (v > best) { best = v; p = i; }
        }
        ipiv[j] = p + 1;
        if (A[IDX(p, j, lda)] != 0.0) {
            if (p != j) {
                for (int c = 0; c < n; ++c) {
                    double t = A[IDX(j, c, lda)];
                    A[IDX(j, c, lda)] = A[IDX(p, c, lda)];
                    A[IDX(p, c, lda)] = t;
                }
            }
            double piv = A[IDX(j, j, lda)];
            for (int i = j + 1; i < m; ++i) A[IDX(i, j, lda)] = A[IDX(i, j, lda)] / piv;
        } else if (info == 0) {
            info = j + 1;
        }
        /* rank-1 update of the trailing block */
        for (int c = j + 1; c < n; ++c) {
            double u = A[IDX(j, c, lda)];
            for (int i = j + 1; i < m; ++i) A[IDX(i, c, lda)] -= A[IDX(i, j, lda)] * u;
        }
    }
    return info;
}

/* Apply row interchanges ipiv[k1..k2) (1-based, absolute rows) to columns
 * [c0, c1) of A, in order (LAPACK dlaswp with increment 1). */
void orc_laswp(double *A, int lda, int c0, int c1, int k1, int k2, const int *ipiv) {
#pragma omp parallel for schedule(static)
    for (int c = c0; c < c1; ++c) {
        for (int k = k1; k < k2; ++k) {
            int p = ipiv[k] - 1;
            if (p != k) {
                double t = A[IDX(k, c, lda)];
                A[IDX(k, c, lda)] = A[IDX(p, c, lda)];
                A[IDX(p, c, lda)] = t;
            }
        }
    }
}

/* B <- L^-1 B for the unit-lower triangle L (nb x nb) of Lm; B is nb x ncol.
 * Column-by-column forward substitution (the "top" block update). */
void orc_trsm_unit_lower(int nb, int ncol, const double *Lm, int ldl, double *B, int ldb) {
#pragma omp parallel for schedule(static)
    for (int c = 0; c < ncol; ++c) {
        for (int k = 0; k < nb; ++k) {
            double xk = B[IDX(k, c, ldb)];
            for (int i = k + 1; i < nb; ++i) B[IDX(i, c, ldb)] -= Lm[IDX(i, k, ldl)] * xk;
        }
    }
}

/* C <- C - A B with A m x k, B k x n, C m x n (the "inner" block update).  Each
 * element accumulates its k products in order of increasing k. */
/* Error-free transformations: s + e = a + b exactly (Knuth's TwoSum), and
 * p + e = a * b exactly (TwoProduct; fma() rounds once, so e is exact). */
static void two_sum(double a, double b, double *s, double *e) {
    const double x = a + b;
    const double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

static void two_prod(double a, double b, double *p, double *e) {
    const double x = a * b;
    *e = fma(a, b, -x);
    *p = x;
}

/* C <- C - A B, each element by Dot2 over the k + 1 terms C(i,j), -A(i,kk) B(kk,j):
 * the running sum s and the compensation c (sum of every rounding error)
 * are added at the end.  The result's error is below
 * u |exact| + gamma_{k+1}^2 (|C| + |A| |B|), gamma_j = j u / (1 - j u). */
void orc_gemm_update_dot2(int m, int n, int k, const double *Am, int lda, const double *Bm, int ldb,
                          double *C, int ldc) {
#pragma omp parallel for schedule(static)
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < m; ++i) {
            double s = C[IDX(i, c, ldc)], comp = 0.0;
            for (int kk = 0; kk < k; ++kk) {
                double p, q, r;
                two_prod(-Am[IDX(i, kk, lda)], Bm[IDX(kk, c, ldb)], &p, &q);
                two_sum(s, p, &s, &r);
                comp += q + r;
            }
            C[IDX(i, c, ldc)] = s + comp;
        }
    }
}

void orc_gemm_update(int m, int n, int k, const double *Am, int lda, const double *Bm, int ldb,
                     double *C, int ldc) {
#pragma omp parallel for schedule(static)
    for (int c = 0; c < n; ++c) {
        for (int kk = 0; kk < k; ++kk) {
            double b = Bm[IDX(kk, c, ldb)];
            const double *a = Am + IDX(0, kk, lda);
            double *cc = C + IDX(0, c, ldc);
            for (int i = 0; i < m; ++i) cc[i] -= a[i] * b;
        }
    }
}

/* The paper's blocked right-looking LU (block width nb), with partial pivoting.
 * ipiv is 1-based and absolute.  Runs the first `ksteps` block iterations
 * (ksteps < 0: all of them); returns info (first zero pivot, 1-based) or 0. */
int orc_getrf_blocked_steps(int n, int nb, double *A, int lda, int *ipiv, int ksteps) {
    int info = 0;
    int step = 0;
    for (int k = 0; k < n; k += nb, ++step) {
        if (ksteps >= 0 && step >= ksteps) break;
        int w = (n - k) < nb ? (n - k) : nb;
        /* 1. panel: rows k..n, columns k..k+w (LU block + left blocks) */
        int pinfo = orc_getf2(n - k, w, A + IDX(k, k, lda), lda, ipiv + k);
        if (pinfo != 0 && info == 0) info = k + pinfo;
        for (int j = k; j < k + w; ++j) ipiv[j] += k;
        /* 2. row interchanges on the columns left and right of the panel */
        orc_laswp(A, lda, 0, k, k, k + w, ipiv);
        orc_laswp(A, lda, k + w, n, k, k + w, ipiv);
        if (k + w < n) {
            /* 3. top blocks: U12 = L11^-1 A12 */
            orc_trsm_unit_lower(w, n - k - w, A + IDX(k, k, lda), lda, A + IDX(k, k + w, lda), lda);
            /* 4. inner blocks: A22 -= L21 U12 */
            orc_gemm_update(n - k - w, n - k - w, w, A + IDX(k + w, k, lda), lda,
                            A + IDX(k, k + w, lda), lda, A + IDX(k + w, k + w, lda), lda);
        }
    }
    return info;
}

int orc_getrf_blocked(int n, int nb, double *A, int lda, int *ipiv) {
    return orc_getrf_blocked_steps(n, nb, A, lda, ipiv, -1);
}

/* The paper's own variant (section "High Performance Linpack": HPL-AI rules,
 * a diagonally dominant A, so the LU needs no pivoting), unblocked: Gaussian
 * elimination without interchanges.  Returns info (first zero pivot) or 0. */
int orc_getf2_nopiv(int m, int n, double *A, int lda) {
    int info = 0;
    int kmax = m < n ? m : n;
    for (int j = 0; j < kmax; ++j) {
        double piv = A[IDX(j, j, lda)];
        if (piv != 0.0) {
            for (int i = j + 1; i < m; ++i) A[IDX(i, j, lda)] = A[IDX(i, j, lda)] / piv;
        } else if (info == 0) {
            info = j + 1;
        }
        for (int c = j + 1; c < n; ++c) {
            double u = A[IDX(j, c, lda)];
            for (int i = j + 1; i < m; ++i) A[IDX(i, c, lda)] -= A[IDX(i, j, lda)] * u;
        }
    }
    return info;
}

/* B <- B U^-1 for the upper triangle U (w x w, non-unit) of Um; B is m x w.
 * Row by row: the paper's "left" block update with U. */
void orc_trsm_right_upper(int m, int w, const double *Um, int ldu, double *B, int ldb) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < w; ++j) {
            double v = B[IDX(i, j, ldb)];
            for (int t = 0; t < j; ++t) v -= B[IDX(i, t, ldb)] * Um[IDX(t, j, ldu)];
            B[IDX(i, j, ldb)] = v / Um[IDX(j, j, ldu)];
        }
    }
}

/* The paper's blocked iteration without pivoting (section "Base
 * Implementation", figure "lu_iteration"): per block, the LU kernel on the
 * diagonal block, the top blocks updated with L (A12 <- L11^-1 A12), the left
 * blocks updated with U (A21 <- A21 U11^-1), and the inner blocks by a matrix
 * multiplication (A22 <- A22 - A21 A12). */
int orc_getrf_nopiv_blocked(int n, int nb, double *A, int lda) {
    int info = 0;
    for (int k = 0; k < n; k += nb) {
        int w = (n - k) < nb ? (n - k) : nb;
        int dinfo = orc_getf2_nopiv(w, w, A + IDX(k, k, lda), lda);
        if (dinfo != 0 && info == 0) info = k + dinfo;
        int rest = n - k - w;
        if (rest > 0) {
            orc_trsm_unit_lower(w, rest, A + IDX(k, k, lda), lda, A + IDX(k, k + w, lda), lda);
            orc_trsm_right_upper(rest, w, A + IDX(k, k, lda), lda, A + IDX(k + w, k, lda), lda);
            orc_gemm_update(rest, rest, w, A + IDX(k + w, k, lda), lda, A + IDX(k, k + w, lda), lda,
                            A + IDX(k + w, k + w, lda), lda);
        }
    }
    return info;
}

/* Unblocked factorization of the whole matrix (the definition). */
int orc_getrf(int n, double *A, int lda, int *ipiv) { return orc_getf2(n, n, A, lda, ipiv); }

/* Solve A X = B from the factors: apply P, then unit-lower forward and upper
 * back substitution.  B (n x nrhs) is overwritten with X. */
void orc_getrs(int n, int nrhs, const double *LU, int lda, const int *ipiv, double *B, int ldb) {
    for (int r = 0; r < nrhs; ++r) {
        double *b = B + IDX(0, r, ldb);
        for (int k = 0; k < n; ++k) {
            int p = ipiv[k] - 1;
            if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
        }
        for (int j = 0; j < n; ++j) {
            double yj = b[j];
            for (int i = j + 1; i < n; ++i) b[i] -= LU[IDX(i, j, lda)] * yj;
        }
        for (int j = n - 1; j >= 0; --j) {
            b[j] = b[j] / LU[IDX(j, j, lda)];
            double xj = b[j];
            for (int i = 0; i < j; ++i) b[i] -= LU[IDX(i, j, lda)] * xj;
        }
    }
}

/* R = B - A X (n x nrhs).  Each r_i sums its products in column order
 * (j = 0, 1, ..., n-1), whatever the number of threads: the threads split the
 * rows, and a block of rows walks every column in order for each right-hand
 * side. */
void orc_residual(int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                  const double *B, int ldb, double *R, int ldr) {
    const int RB = 256;
#pragma omp parallel for schedule(static)
    for (int i0 = 0; i0 < n; i0 += RB) {
        const int i1 = (i0 + RB) < n ? (i0 + RB) : n;
        for (int r = 0; r < nrhs; ++r)
            for (int i = i0; i < i1; ++i) R[IDX(i, r, ldr)] = B[IDX(i, r, ldb)];
        for (int j = 0; j < n; ++j) {
            const double *a = A + IDX(0, j, lda);
            for (int r = 0; r < nrhs; ++r) {
                const double xj = X[IDX(j, r, ldx)];
                double *rr = R + IDX(0, r, ldr);
                for (int i = i0; i < i1; ++i) rr[i] -= a[i] * xj;
            }
        }
    }
}

/* ||A||_inf: the largest absolute row sum of an m x n matrix. */
double orc_norm_inf_mat(int m, int n, const double *A, int lda) {
    double *rs = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < m; ++i) rs[i] += fabs(A[IDX(i, j, lda)]);
    double mx = 0.0;
    for (int i = 0; i < m; ++i) if (rs[i] > mx) mx = rs[i];
    free(rs);
    return mx;
}

/* ||A||_1: the largest absolute column sum. */
double orc_norm_one_mat(int m, int n, const double *A, int lda) {
    double mx = 0.0;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += fabs(A[IDX(i, j, lda)]);
        if (s > mx) mx = s;
    }
    return mx;
}

double orc_norm_inf_vec(int n, const double *x) {
    double mx = 0.0;
    for (int i = 0; i < n; ++i) if (fabs(x[i]) > mx) mx = fabs(x[i]);
    return mx;
}

/* HPL scaled residual of one right-hand side, with eps the unit roundoff 2^-53. */
double orc_scaled_residual(int n, double rnorm, double anorm, double xnorm, double bnorm) {
    const double eps = ldexp(1.0, -53);
    return rnorm / (eps * (anorm * xnorm + bnorm) * (double)n);
}

/* The paper-shaped normalized residual ||r||_inf / (n ||b||_inf eps), eps = 2^-53. */
double orc_paper_residual(int n, double rnorm, double bnorm) {
    const double eps = ldexp(1.0, -53);
    return rnorm / ((double)n * bnorm * eps);
}

/* x <- A^-T x from the factors P A = L U:  A^T = U^T L^T P, so solve U^T w = x,
 * L^T v = w, then x = P^T v (undo the interchanges in reverse order). */
static void orc_getrs_trans(int n, const double *LU, int lda, const int *ipiv, double *x) {
    for (int j = 0; j < n; ++j) {
        double s = x[j];
        for (int i = 0; i < j; ++i) s -= LU[IDX(i, j, lda)] * x[i];
        x[j] = s / LU[IDX(j, j, lda)];
    }
    for (int j = n - 1; j >= 0; --j) {
        double s = x[j];
        for (int i = j + 1; i < n; ++i) s -= LU[IDX(i, j, lda)] * x[i];
        x[j] = s;
    }
    for (int k = n - 1; k >= 0; --k) {
        int p = ipiv[k] - 1;
        if (p != k) { double t = x[k]; x[k] = x[p]; x[p] = t; }
    }
}

/* Estimate of ||A^-1||_1 (Hager 1984, Higham 1988 Algorithm 4.1), then
 * kappa_1 estimate = anorm1 * that.  Returns the kappa_1 estimate. */
double orc_cond1_est(int n, const double *LU, int lda, const int *ipiv, double anorm1) {
    if (n <= 0) return 0.0;
    double *x = (double *)malloc(sizeof(double) * (size_t)n);
    double *xi = (double *)malloc(sizeof(double) * (size_t)n);
    double *z = (double *)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i) x[i] = 1.0 / (double)n;
    double est = 0.0;
    int jlast = -1;
    for (int iter = 0; iter < 5; ++iter) {
        /* x <- A^-1 x */
        memcpy(z, x, sizeof(double) * (size_t)n);
        orc_getrs(n, 1, LU, lda, ipiv, z, n);
        memcpy(x, z, sizeof(double) * (size_t)n);
        double gamma = 0.0;
        for (int i = 0; i < n; ++i) gamma += fabs(x[i]);
        int same_sign = iter > 0;
        for (int i = 0; i < n; ++i) {
            double s = x[i] >= 0.0 ? 1.0 : -1.0;
            if (iter > 0 && s != xi[i]) same_sign = 0;
            xi[i] = s;
        }
        if (iter > 0 && (same_sign || gamma <= est)) { if (gamma > est) est = gamma; break; }
        est = gamma;
        /* z <- A^-T xi */
        memcpy(z, xi, sizeof(double) * (size_t)n);
        orc_getrs_trans(n, LU, lda, ipiv, z);
        int j = 0;
        double zmax = fabs(z[0]);
        for (int i = 1; i < n; ++i) if (fabs(z[i]) > zmax) { zmax = fabs(z[i]); j = i; }
        if (iter > 0 && j == jlast) break;
        jlast = j;
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        x[j] = 1.0;
    }
    /* Higham's extra test vector b_i = (-1)^i (1 + i/(n-1)) */
    for (int i = 0; i < n; ++i)
        x[i] = ((i & 1) ? -1.0 : 1.0) * (1.0 + (n > 1 ? (double)i / (double)(n - 1) : 0.0));
    orc_getrs(n, 1, LU, lda, ipiv, x, n);
    double alt = 0.0;
    for (int i = 0; i < n; ++i) alt += fabs(x[i]);
    alt = 2.0 * alt / (3.0 * (double)n);
    if (alt > est) est = alt;
    free(x); free(xi); free(z);
    return est * anorm1;
}

/* Round-to-nearest-even of FP32 values to bfloat16 (8 significant bits) and
 * to IEEE binary16 (11 significant bits, with subnormals and overflow to inf),
 * returned as the exact FP64 value of the 16-bit result. */
void orc_round_bf16(int64_t count, const float *in, double *out) {
    for (int64_t t = 0; t < count; ++t) {
        float f = in[t];
        uint32_t u;
        memcpy(&u, &f, 4);
        if ((u & 0x7f800000u) == 0x7f800000u) { out[t] = (double)f; continue; }
        uint32_t lsb = (u >> 16) & 1u;
        u = (u + 0x7fffu + lsb) & 0xffff0000u;
        float r;
        memcpy(&r, &u, 4);
        out[t] = (double)r;
    }
}

void orc_round_fp16(int64_t count, const float *in, double *out) {
    for (int64_t t = 0; t < count; ++t) {
        double v = (double)in[t];
        if (isnan(v) || isinf(v)) { out[t] = v; continue; }
        double a = fabs(v);
        double q;
        if (a < ldexp(1.0, -14)) {
            q = ldexp(1.0, -24);            /* subnormal spacing */
        } else {
            int e;
            frexp(a, &e);                   /* a = f 2^e, f in [0.5, 1) */
            q = ldexp(1.0, (e - 1) - 10);   /* spacing of 11-bit significands */
        }
        double k = a / q;                   /* exact: a is a multiple of 2^-149 */
        double fl = floor(k);
        double rem = k - fl;
        double kr = fl;
        if (rem > 0.5 || (rem == 0.5 && fmod(fl, 2.0) != 0.0)) kr = fl + 1.0;
        double r = kr * q;
        if (r > 65504.0) r = INFINITY;
        out[t] = v < 0 ? -r : r;
    }
}
