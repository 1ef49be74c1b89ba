/*
 * CPU oracle for Frobenius inversion (Dai, Lim and Ye, "Complex matrix
 * inversion via real matrix inversions").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code with the CUDA path.
 *
 * Plain, slow, FP64.  Every routine follows one algorithm of the paper in the
 * paper's order and notation; there is no blocking, fusion or reordering.
 * OpenMP is used only across independent right-hand sides / rows, which does
 * not change the arithmetic of any single entry.
 *
 * Storage: n x n matrices, row-major, leading dimension n.  Complex matrices
 * are interleaved (re, im) pairs of double, i.e. C99 double complex.
 *
 * Return codes: 0 on success; k > 0 when the k-th (1-based) pivot of a
 * factorisation is exactly zero or not finite (LU) or the k-th Cholesky
 * diagonal is not positive (Cholesky); -1 on allocation failure; -2 on a bad
 * argument.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ORC_MUTANT plants one deliberate mistake (k = 1..15) so that a test can check
 * that the pins catch it.  Product builds of the oracle use ORC_MUTANT = 0. */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

typedef double complex zc;

#define IDX(i, j) ((size_t)(i) * (size_t)n + (size_t)(j))

static double abs2(zc z) { return creal(z) * creal(z) + cimag(z) * cimag(z); }

/* ------------------------------------------------------------------------- */
/* Complex LU with partial pivoting: X = P^T L U  (Algorithm LU1, step 1).    */
/* In place: strictly lower part holds L (unit diagonal), upper part U.       */
/* piv[k] = row exchanged with row k at step k.  The pivot is the entry of    */
/* largest modulus (compared as |re|^2+|im|^2); ties go to the lowest row.    */
/* ------------------------------------------------------------------------- */
static int zgetrf_plain(int n, zc *a, int *piv)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = abs2(a[IDX(k, k)]);
        for (int i = k + 1; i < n; ++i) {
            double v = abs2(a[IDX(i, k)]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (!(best > 0.0) || !isfinite(best)) return k + 1;
        if (p != k)
            for (int j = 0; j < n; ++j) { zc t = a[IDX(k, j)]; a[IDX(k, j)] = a[IDX(p, j)]; a[IDX(p, j)] = t; }
        zc d = a[IDX(k, k)];
        for (int i = k + 1; i < n; ++i) a[IDX(i, k)] /= d;
#pragma omp parallel for schedule(static)
        for (int i = k + 1; i < n; ++i) {
            zc l = a[IDX(i, k)];
            for (int j = k + 1; j < n; ++j) a[IDX(i, j)] -= l * a[IDX(k, j)];
        }
    }
    return 0;
}

/* Real LU with partial pivoting, same conventions (Algorithm 4, steps 1, 4). */
static int dgetrf_plain(int n, double *a, int *piv)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[IDX(k, k)]);
        for (int i = k + 1; i < n; ++i) {
            double v = fabs(a[IDX(i, k)]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (!(best > 0.0) || !isfinite(best)) return k + 1;
        if (p != k)
            for (int j = 0; j < n; ++j) { double t = a[IDX(k, j)]; a[IDX(k, j)] = a[IDX(p, j)]; a[IDX(p, j)] = t; }
        double d = a[IDX(k, k)];
        for (int i = k + 1; i < n; ++i) a[IDX(i, k)] /= d;
#pragma omp parallel for schedule(static)
        for (int i = k + 1; i < n; ++i) {
            double l = a[IDX(i, k)];
            for (int j = k + 1; j < n; ++j) a[IDX(i, j)] -= l * a[IDX(k, j)];
        }
    }
    return 0;
}

/* Column permutation Y <- Y P for P X = L U with the swaps of piv, i.e. the
 * swaps applied to columns in reverse order (Algorithm LU1, output step). */
static void zcolperm(int n, zc *y, const int *piv)
{
    if (ORC_MUTANT == 7) { /* planted: forward order */
        for (int k = 0; k < n; ++k) {
            int p = piv[k];
            if (p != k)
                for (int i = 0; i < n; ++i) { zc t = y[IDX(i, k)]; y[IDX(i, k)] = y[IDX(i, p)]; y[IDX(i, p)] = t; }
        }
        return;
    }
    for (int k = n - 1; k >= 0; --k) {
        int p = piv[k];
        if (p != k)
            for (int i = 0; i < n; ++i) { zc t = y[IDX(i, k)]; y[IDX(i, k)] = y[IDX(i, p)]; y[IDX(i, p)] = t; }
    }
}
static void dcolperm(int n, double *y, const int *piv)
{
    for (int k = n - 1; k >= 0; --k) {
        int p = piv[k];
        if (p != k)
            for (int i = 0; i < n; ++i) { double t = y[IDX(i, k)]; y[IDX(i, k)] = y[IDX(i, p)]; y[IDX(i, p)] = t; }
    }
}

/* ------------------------------------------------------------------------- */
/* Algorithm LU1: complex inversion by LU.                                    */
/* left = 1: the paper's order. U X1 = I (backward), X2 L = X1 (forward),     */
/*           X^{-1} = X2 P.  This is a left inverse (Y X = I).                */
/* left = 0: the right-inverse variant the paper mentions after Algorithm     */
/*           LU1: swap the substitutions, i.e. solve L U y_j = P e_j.         */
/* ------------------------------------------------------------------------- */
int orc_cplx_lu_inv(int n, const zc *m, zc *x, int left)
{
    if (n < 1) return -2;
    zc *a = malloc(sizeof(zc) * (size_t)n * n);
    int *piv = malloc(sizeof(int) * (size_t)n);
    if (!a || !piv) { free(a); free(piv); return -1; }
    memcpy(a, m, sizeof(zc) * (size_t)n * n);
    int info = zgetrf_plain(n, a, piv);
    if (info) { free(a); free(piv); return info; }

    if (left) {
        /* X1 = U^{-1}: backward substitution U X1 = I, one column at a time. */
        zc *x1 = calloc((size_t)n * n, sizeof(zc));
        if (!x1) { free(a); free(piv); return -1; }
#pragma omp parallel for schedule(dynamic, 4)
        for (int j = 0; j < n; ++j) {
            for (int i = n - 1; i >= 0; --i) {
                zc s = (i == j) ? 1.0 : 0.0;
                for (int k = i + 1; k < n; ++k) s -= a[IDX(i, k)] * x1[IDX(k, j)];
                x1[IDX(i, j)] = s / a[IDX(i, i)];
            }
        }
        /* X2 L = X1: forward substitution along each row of X2, starting
         * from the last column because L is unit lower triangular. */
#pragma omp parallel for schedule(static)
        for (int r = 0; r < n; ++r) {
            for (int j = n - 1; j >= 0; --j) {
                zc s = x1[IDX(r, j)];
                for (int i = j + 1; i < n; ++i) s -= x[IDX(r, i)] * a[IDX(i, j)];
                x[IDX(r, j)] = s;
            }
        }
        free(x1);
        zcolperm(n, x, piv);
    } else {
        /* Right inverse: the columns of P, then L z = P e_j, then U y = z. */
        for (size_t t = 0; t < (size_t)n * n; ++t) x[t] = 0.0;
        int *perm = malloc(sizeof(int) * (size_t)n);
        if (!perm) { free(a); free(piv); return -1; }
        for (int i = 0; i < n; ++i) perm[i] = i;
        for (int k = 0; k < n; ++k) { int t = perm[k]; perm[k] = perm[piv[k]]; perm[piv[k]] = t; }
        /* (P I)[i, perm[i]] = 1 */
        for (int i = 0; i < n; ++i) x[IDX(i, perm[i])] = 1.0;
        free(perm);
#pragma omp parallel for schedule(dynamic, 4)
        for (int j = 0; j < n; ++j) {
            for (int i = 0; i < n; ++i) {
                zc s = x[IDX(i, j)];
                for (int k = 0; k < i; ++k) s -= a[IDX(i, k)] * x[IDX(k, j)];
                x[IDX(i, j)] = s;
            }
            for (int i = n - 1; i >= 0; --i) {
                zc s = x[IDX(i, j)];
                for (int k = i + 1; k < n; ++k) s -= a[IDX(i, k)] * x[IDX(k, j)];
                x[IDX(i, j)] = s / a[IDX(i, i)];
            }
        }
    }
    free(a);
    free(piv);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Algorithm Cholesky2: complex HPD inversion.  A = R^H R with R upper        */
/* triangular; R^H X1 = I; R X2 = X1; A^{-1} = X2.  Only the lower triangle   */
/* of m is read (the upper one is taken as its conjugate transpose); the      */
/* imaginary parts of the diagonal are ignored.                               */
/* ------------------------------------------------------------------------- */
int orc_cplx_chol_inv(int n, const zc *m, zc *x)
{
    if (n < 1) return -2;
    zc *r = calloc((size_t)n * n, sizeof(zc));
    if (!r) return -1;
    for (int j = 0; j < n; ++j) {
        /* a_jj is real for Hermitian input */
        double d = creal(m[IDX(j, j)]);
        for (int k = 0; k < j; ++k) d -= abs2(r[IDX(k, j)]);
        if (!(d > 0.0) || !isfinite(d)) { free(r); return j + 1; }
        double rjj = sqrt(d);
        r[IDX(j, j)] = rjj;
#pragma omp parallel for schedule(static)
        for (int i = j + 1; i < n; ++i) {
            zc s = conj(m[IDX(i, j)]); /* a_ji from the lower triangle */
            for (int k = 0; k < j; ++k) s -= (ORC_MUTANT == 4 ? r[IDX(k, j)] : conj(r[IDX(k, j)])) * r[IDX(k, i)];
            r[IDX(j, i)] = s / rjj;
        }
    }
    /* R^H X1 = I (R^H lower: substitute from the top), then R X2 = X1. */
#pragma omp parallel for schedule(dynamic, 4)
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) {
            zc s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= conj(r[IDX(k, i)]) * x[IDX(k, c)];
            x[IDX(i, c)] = s / r[IDX(i, i)];
        }
        for (int i = n - 1; i >= 0; --i) {
            zc s = x[IDX(i, c)];
            for (int k = i + 1; k < n; ++k) s -= r[IDX(i, k)] * x[IDX(k, c)];
            x[IDX(i, c)] = s / r[IDX(i, i)];
        }
    }
    free(r);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Real building blocks for the Frobenius routines.                           */
/* ------------------------------------------------------------------------- */

/* Solve L U X = P C for all columns of C (in place in c), from dgetrf_plain. */
static void dlu_solve_cols(int n, const double *lu, const int *piv, double *c)
{
    for (int k = 0; k < n; ++k) {
        int p = piv[k];
        if (p != k)
            for (int j = 0; j < n; ++j) { double t = c[IDX(k, j)]; c[IDX(k, j)] = c[IDX(p, j)]; c[IDX(p, j)] = t; }
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < n; ++i) {
            double s = c[IDX(i, j)];
            for (int k = 0; k < i; ++k) s -= lu[IDX(i, k)] * c[IDX(k, j)];
            c[IDX(i, j)] = s;
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = c[IDX(i, j)];
            for (int k = i + 1; k < n; ++k) s -= lu[IDX(i, k)] * c[IDX(k, j)];
            c[IDX(i, j)] = s / lu[IDX(i, i)];
        }
    }
}

/* Solve Y (P^T L U) = C for all rows of C (in place): first W U = C, then
 * V L = W, then Y = V P (column swaps in reverse order). */
static void dlu_solve_rows(int n, const double *lu, const int *piv, double *c)
{
#pragma omp parallel for schedule(static)
    for (int r = 0; r < n; ++r) {
        for (int j = 0; j < n; ++j) {
            double s = c[IDX(r, j)];
            for (int i = 0; i < j; ++i) s -= c[IDX(r, i)] * lu[IDX(i, j)];
            c[IDX(r, j)] = s / lu[IDX(j, j)];
        }
        for (int j = n - 1; j >= 0; --j) {
            double s = c[IDX(r, j)];
            for (int i = j + 1; i < n; ++i) s -= c[IDX(r, i)] * lu[IDX(i, j)];
            c[IDX(r, j)] = s;
        }
    }
    dcolperm(n, c, piv);
}

/* C = D + A B (plain triple loop); D may be NULL for C = A B. */
static void dgemm_plain(int n, const double *a, const double *b, const double *d, double *c)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += a[IDX(i, k)] * b[IDX(k, j)];
            c[IDX(i, j)] = d ? d[IDX(i, j)] + s : s;
        }
}

/* Real inverse of a (n x n) by LU: A^{-1} = U^{-1} L^{-1} P, computed as the
 * right inverse (solve with the identity). */
static int dinv_plain(int n, const double *a, double *ainv)
{
    double *lu = malloc(sizeof(double) * (size_t)n * n);
    int *piv = malloc(sizeof(int) * (size_t)n);
    if (!lu || !piv) { free(lu); free(piv); return -1; }
    memcpy(lu, a, sizeof(double) * (size_t)n * n);
    int info = dgetrf_plain(n, lu, piv);
    if (!info) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) ainv[IDX(i, j)] = (i == j) ? 1.0 : 0.0;
        dlu_solve_cols(n, lu, piv, ainv);
    }
    free(lu);
    free(piv);
    return info;
}

static void split_planes(int n, const zc *m, double *a, double *b)
{
    for (size_t t = 0; t < (size_t)n * n; ++t) { a[t] = creal(m[t]); b[t] = cimag(m[t]); }
}

/* ------------------------------------------------------------------------- */
/* Algorithm "Frobenius inversion" over C = R[xi], xi^2 = -1 (tau = 1):       */
/* X1 = A^{-1}; X2 = X1 B; X3 = B X2; X4 = A + X3; X5 = X4^{-1};              */
/* X6 = X2 X5; result X5 - i X6.  Explicit real inversions, as written.       */
/* stage != NULL receives X2 (= A^{-1}B), X4 (= S) and X5 (= S^{-1}).         */
/* ------------------------------------------------------------------------- */
int orc_frob_inv_basic(int n, const zc *m, zc *x, double *x2_out, double *s_out, double *sinv_out)
{
    if (n < 1) return -2;
    size_t nn = (size_t)n * n;
    double *w = malloc(sizeof(double) * nn * 7);
    if (!w) return -1;
    double *A = w, *B = w + nn, *X1 = w + 2 * nn, *X2 = w + 3 * nn, *X4 = w + 4 * nn, *X5 = w + 5 * nn,
           *X6 = w + 6 * nn;
    split_planes(n, m, A, B);
    int info = dinv_plain(n, A, X1);
    if (info) { free(w); return info; }
    dgemm_plain(n, X1, B, NULL, X2);   /* X2 = A^{-1} B          */
    dgemm_plain(n, B, X2, A, X4);      /* X4 = A + B X2  (tau=1) */
    info = dinv_plain(n, X4, X5);      /* X5 = X4^{-1}           */
    if (info) { free(w); return info; }
    if (ORC_MUTANT == 1) dgemm_plain(n, X5, X2, NULL, X6); /* planted: X5 X2 */
    else dgemm_plain(n, X2, X5, NULL, X6);  /* X6 = X2 X5             */
    for (size_t t = 0; t < nn; ++t) x[t] = X5[t] - I * X6[t];
    if (x2_out) memcpy(x2_out, X2, sizeof(double) * nn);
    if (s_out) memcpy(s_out, X4, sizeof(double) * nn);
    if (sinv_out) memcpy(sinv_out, X5, sizeof(double) * nn);
    free(w);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The formula for invertible B (Sec. 4.2, before Lemma "rand Frob"):         */
/* (A + iB)^{-1} = B^{-1} A (A B^{-1} A + B)^{-1} - i (A B^{-1} A + B)^{-1}.  */
/* Y1 = B^{-1}; Y2 = Y1 A; T = B + A Y2; Y5 = T^{-1}; Y6 = Y2 Y5;             */
/* result Y6 - i Y5.  Explicit real inversions, as written.                   */
/* ------------------------------------------------------------------------- */
int orc_frob_inv_b(int n, const zc *m, zc *x)
{
    if (n < 1) return -2;
    size_t nn = (size_t)n * n;
    double *w = malloc(sizeof(double) * nn * 7);
    if (!w) return -1;
    double *A = w, *B = w + nn, *Y1 = w + 2 * nn, *Y2 = w + 3 * nn, *T = w + 4 * nn, *Y5 = w + 5 * nn,
           *Y6 = w + 6 * nn;
    split_planes(n, m, A, B);
    int info = dinv_plain(n, B, Y1);
    if (info) { free(w); return info; }
    dgemm_plain(n, Y1, A, NULL, Y2);   /* Y2 = B^{-1} A          */
    dgemm_plain(n, A, Y2, B, T);       /* T = B + A B^{-1} A     */
    info = dinv_plain(n, T, Y5);       /* Y5 = T^{-1}            */
    if (info) { free(w); return info; }
    dgemm_plain(n, Y2, Y5, NULL, Y6);  /* Y6 = B^{-1} A T^{-1}   */
    for (size_t t = 0; t < nn; ++t) x[t] = Y6[t] - (ORC_MUTANT == 14 ? -1.0 : 1.0) * I * Y5[t];
    free(w);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Bicomplex matrices (the iterated quadratic extension of Sec. 2.4 with     */
/* m = 2, xi_1^2 = xi_2^2 = -1; written X = A + jB with A, B complex and j   */
/* commuting with i).  The map A + jB -> [[A, -B], [B, A]] is an injective   */
/* algebra homomorphism into 2n x 2n complex matrices (j^2 = -1 matches the  */
/* block structure), so X^{-1} = Y0 + jY1 is read off the inverse of the     */
/* embedding, [[Y0, -Y1], [Y1, Y0]].  The inverse by complex LU.              */
/* ------------------------------------------------------------------------- */
int orc_bicomplex_inv(int n, const zc *a, const zc *b, zc *y0, zc *y1)
{
    if (n < 1) return -2;
    const int n2 = 2 * n;
    zc *e = malloc(sizeof(zc) * (size_t)n2 * n2), *ei = malloc(sizeof(zc) * (size_t)n2 * n2);
    if (!e || !ei) { free(e); free(ei); return -1; }
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const zc av = a[(size_t)i * n + k], bv = b[(size_t)i * n + k];
            e[(size_t)i * n2 + k] = av;
            e[(size_t)i * n2 + n + k] = -bv;
            e[(size_t)(n + i) * n2 + k] = bv;
            e[(size_t)(n + i) * n2 + n + k] = av;
        }
    int info = orc_cplx_lu_inv(n2, e, ei, 0);
    if (info == 0)
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < n; ++k) {
                y0[(size_t)i * n + k] = ei[(size_t)i * n2 + k];
                y1[(size_t)i * n + k] = (ORC_MUTANT == 15 ? -1.0 : 1.0) * ei[(size_t)(n + i) * n2 + k];
            }
    free(e);
    free(ei);
    return info;
}

/* ------------------------------------------------------------------------- */
/* Algorithm "Frobenius inversion with LU decomposition":                     */
/* A = P1^T L1 U1; L1 U1 X1 = P1 B; X2 = A + B X1; X2 = P2^T L2 U2;           */
/* [X3, X4] P2^T L2 U2 = [I, X1] (right division); result X3 - i X4.         */
/* ------------------------------------------------------------------------- */
static int frob_lu_planes(int n, const double *A, const double *B, double *X3, double *X4)
{
    size_t nn = (size_t)n * n;
    double *w = malloc(sizeof(double) * nn * 3);
    int *piv = malloc(sizeof(int) * (size_t)n);
    if (!w || !piv) { free(w); free(piv); return -1; }
    double *LU = w, *X1 = w + nn, *X2 = w + 2 * nn;
    memcpy(LU, A, sizeof(double) * nn);
    int info = dgetrf_plain(n, LU, piv);                   /* step 1 */
    if (info) { free(w); free(piv); return info; }
    memcpy(X1, B, sizeof(double) * nn);
    dlu_solve_cols(n, LU, piv, X1);                        /* step 2 */
    dgemm_plain(n, B, X1, ORC_MUTANT == 3 ? NULL : A, X2); /* step 3 */
    info = dgetrf_plain(n, X2, piv);                       /* step 4 */
    if (info) { free(w); free(piv); return info; }
    for (int i = 0; i < n; ++i)                            /* step 5 */
        for (int j = 0; j < n; ++j) X3[IDX(i, j)] = (i == j) ? 1.0 : 0.0;
    dlu_solve_rows(n, X2, piv, X3);
    memcpy(X4, X1, sizeof(double) * nn);
    dlu_solve_rows(n, X2, piv, X4);
    free(w);
    free(piv);
    return 0;
}

int orc_frob_inv_lu(int n, const zc *m, zc *x)
{
    if (n < 1) return -2;
    size_t nn = (size_t)n * n;
    double *w = malloc(sizeof(double) * nn * 4);
    if (!w) return -1;
    double *A = w, *B = w + nn, *X3 = w + 2 * nn, *X4 = w + 3 * nn;
    split_planes(n, m, A, B);
    int info = frob_lu_planes(n, A, B, X3, X4);
    if (!info)
        for (size_t t = 0; t < nn; ++t) x[t] = X3[t] - (ORC_MUTANT == 2 ? -1.0 : 1.0) * I * X4[t];
    free(w);
    return info;
}

/* ------------------------------------------------------------------------- */
/* Algorithm "Almost sure Frobenius inversion", with mu given by the caller:  */
/* X1 = A - mu B; X2 = mu A + B; X3 + i X4 = (X1 + i X2)^{-1} by Frobenius    */
/* inversion with LU; X5 = X3 - mu X4; X6 = mu X3 + X4; result X5 + i X6.     */
/* Here X4 is the imaginary part of the inner inverse.                        */
/* ------------------------------------------------------------------------- */
int orc_frob_inv_rand(int n, const zc *m, double mu, zc *x)
{
    if (n < 1) return -2;
    size_t nn = (size_t)n * n;
    double *w = malloc(sizeof(double) * nn * 6);
    if (!w) return -1;
    double *A = w, *B = w + nn, *X1 = w + 2 * nn, *X2 = w + 3 * nn, *R = w + 4 * nn, *Q = w + 5 * nn;
    split_planes(n, m, A, B);
    for (size_t t = 0; t < nn; ++t) { X1[t] = A[t] - mu * B[t]; X2[t] = mu * A[t] + B[t]; }
    int info = frob_lu_planes(n, X1, X2, R, Q); /* inverse = R - i Q */
    if (!info)
        for (size_t t = 0; t < nn; ++t) {
            double X3 = R[t], X4 = -Q[t];
            x[t] = (ORC_MUTANT == 6 ? X3 + mu * X4 : X3 - mu * X4) + I * (mu * X3 + X4);
        }
    free(w);
    return info;
}

/* Real Cholesky A = R^T R, R upper; returns j+1 if the j-th diagonal is not
 * positive. */
static int dpotrf_plain(int n, const double *a, double *r)
{
    for (size_t t = 0; t < (size_t)n * n; ++t) r[t] = 0.0;
    for (int j = 0; j < n; ++j) {
        double d = a[IDX(j, j)];
        for (int k = 0; k < j; ++k) d -= r[IDX(k, j)] * r[IDX(k, j)];
        if (!(d > 0.0) || !isfinite(d)) return j + 1;
        double rjj = sqrt(d);
        r[IDX(j, j)] = rjj;
#pragma omp parallel for schedule(static)
        for (int i = j + 1; i < n; ++i) {
            double s = a[IDX(j, i)];
            for (int k = 0; k < j; ++k) s -= r[IDX(k, j)] * r[IDX(k, i)];
            r[IDX(j, i)] = s / rjj;
        }
    }
    return 0;
}

/* R^T Y = C (R^T lower: from the top), all columns, in place. */
static void dtrsm_rt(int n, const double *r, double *c)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double s = c[IDX(i, j)];
            for (int k = 0; k < i; ++k) s -= r[IDX(k, i)] * c[IDX(k, j)];
            c[IDX(i, j)] = s / r[IDX(i, i)];
        }
}
/* R Y = C (R upper: from the bottom), all columns, in place. */
static void dtrsm_r(int n, const double *r, double *c)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < n; ++j)
        for (int i = n - 1; i >= 0; --i) {
            double s = c[IDX(i, j)];
            for (int k = i + 1; k < n; ++k) s -= r[IDX(i, k)] * c[IDX(k, j)];
            c[IDX(i, j)] = s / r[IDX(i, i)];
        }
}

/* ------------------------------------------------------------------------- */
/* Algorithm "Frobenius inversion with Cholesky decomposition" (HPD input):   */
/* A = R1^T R1; R1^T X1 = B; R1 X2 = X1; X3 = X1^T X1; X4 = A - X3;           */
/* X4 = R2^T R2; R2^T X5 = I; R2 X6 = X5; X7 = X2 X6; result X6 - i X7.       */
/* A is the symmetric part read from the lower triangle of m; B is the skew   */
/* part read from the strictly lower triangle (diagonal of B taken as 0).     */
/* Returns k > 0 if A (k <= n) or S (k = n + j) is not positive definite.     */
/* ------------------------------------------------------------------------- */
int orc_frob_inv_chol(int n, const zc *m, zc *x)
{
    if (n < 1) return -2;
    size_t nn = (size_t)n * n;
    double *w = malloc(sizeof(double) * nn * 7);
    if (!w) return -1;
    double *A = w, *B = w + nn, *R1 = w + 2 * nn, *X1 = w + 3 * nn, *X2 = w + 4 * nn, *X4 = w + 5 * nn,
           *X7 = w + 6 * nn;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            zc v = m[IDX(i, j)];
            A[IDX(i, j)] = A[IDX(j, i)] = creal(v);
            B[IDX(i, j)] = (i == j) ? 0.0 : cimag(v);
            B[IDX(j, i)] = (i == j) ? 0.0 : -cimag(v);
        }
    int info = dpotrf_plain(n, A, R1);                       /* step 1 */
    if (info) { free(w); return info; }
    memcpy(X1, B, sizeof(double) * nn);
    dtrsm_rt(n, R1, X1);                                      /* step 2 */
    memcpy(X2, X1, sizeof(double) * nn);
    dtrsm_r(n, R1, X2);                                       /* step 3 */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)                               /* steps 4-5 */
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k)
                s += ORC_MUTANT == 5 ? X1[IDX(i, k)] * X1[IDX(j, k)] : X1[IDX(k, i)] * X1[IDX(k, j)];
            X4[IDX(i, j)] = A[IDX(i, j)] - s;
        }
    double *R2 = R1; /* R1 is no longer needed */
    info = dpotrf_plain(n, X4, R2);                           /* step 6 */
    if (info) { free(w); return n + info; }
    double *X6 = X1; /* X1 is no longer needed */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) X6[IDX(i, j)] = (i == j) ? 1.0 : 0.0;
    dtrsm_rt(n, R2, X6);                                      /* step 7 */
    dtrsm_r(n, R2, X6);                                       /* step 8 */
    dgemm_plain(n, X2, X6, NULL, X7);                         /* step 9 */
    for (size_t t = 0; t < nn; ++t) x[t] = X6[t] - I * X7[t];
    free(w);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Closed forms.                                                              */
/* ------------------------------------------------------------------------- */

/* [[a, b], [c, d]]^{-1} = (ad - bc)^{-1} [[d, -b], [-c, a]]. */
int orc_inv2x2(const zc *m, zc *x)
{
    zc det = m[0] * m[3] - m[1] * m[2];
    if (det == 0.0) return 1;
    x[0] = m[3] / det;
    x[1] = -m[1] / det;
    x[2] = -m[2] / det;
    x[3] = m[0] / det;
    return 0;
}

/* Determinant by Laplace expansion along the first row (n <= 4). */
static zc zdet_laplace(int n, const zc *a)
{
    if (n == 1) return a[0];
    zc minor[16];
    zc det = 0.0;
    for (int c = 0; c < n; ++c) {
        int t = 0;
        for (int i = 1; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (j != c) minor[t++] = a[(size_t)i * n + j];
        zc cof = ((c & 1) ? -1.0 : 1.0) * zdet_laplace(n - 1, minor);
        det += a[c] * cof;
    }
    return det;
}

/* X = adj(M) / det(M), adj(M)[i][j] = (-1)^{i+j} det(M with row j and
 * column i removed).  Brute force for n <= 4. */
int orc_adjugate_inv(int n, const zc *m, zc *x)
{
    if (n < 1 || n > 4) return -2;
    zc det = zdet_laplace(n, m);
    if (det == 0.0) return 1;
    if (n == 1) { x[0] = 1.0 / m[0]; return 0; }
    zc minor[16];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            int t = 0;
            for (int r = 0; r < n; ++r) {
                if (r == j) continue;
                for (int c = 0; c < n; ++c)
                    if (c != i) minor[t++] = m[(size_t)r * n + c];
            }
            zc cof = (((i + j) & 1) ? -1.0 : 1.0) * zdet_laplace(n - 1, minor);
            x[(size_t)i * n + j] = cof / det;
        }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of inversion: for X = M^{-1} and a real loss with gradient G with  */
/* respect to X (G = dL/dRe X + i dL/dIm X), the gradient with respect to M   */
/* is -X^H G X^H, from d(M^{-1}) = -M^{-1} dM M^{-1}.  Plain triple loops.    */
/* ------------------------------------------------------------------------- */
int orc_inv_adjoint(int n, const zc *x, const zc *g, zc *out)
{
    if (n < 1) return -2;
    zc *p = malloc(sizeof(zc) * (size_t)n * n);
    if (!p) return -1;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)          /* P = X^H G */
        for (int j = 0; j < n; ++j) {
            zc s = 0.0;
            for (int k = 0; k < n; ++k) s += (ORC_MUTANT == 8 ? x[IDX(k, i)] : conj(x[IDX(k, i)])) * g[IDX(k, j)];
            p[IDX(i, j)] = s;
        }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)          /* out = -P X^H */
        for (int j = 0; j < n; ++j) {
            zc s = 0.0;
            for (int k = 0; k < n; ++k) s += p[IDX(i, k)] * conj(x[IDX(j, k)]);
            out[IDX(i, j)] = -s;
        }
    free(p);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Newton iteration for the matrix sign function (Sec. 5.3, eq. "iter"):      */
/* X_{k+1} = (X_k + X_k^{-1}) / 2, X_0 = M, a fixed number of steps, each     */
/* inverse by complex LU (right inverse).                                     */
/* ------------------------------------------------------------------------- */
int orc_sign_newton(int n, const zc *m, int iters, zc *out)
{
    if (n < 1 || iters < 0) return -2;
    size_t nn = (size_t)n * n;
    zc *xi = malloc(sizeof(zc) * nn);
    if (!xi) return -1;
    memcpy(out, m, sizeof(zc) * nn);
    for (int k = 0; k < iters; ++k) {
        int info = orc_cplx_lu_inv(n, out, xi, 0);
        if (info) { free(xi); return info; }
        for (size_t t = 0; t < nn; ++t) out[t] = (ORC_MUTANT == 9 ? 1.0 : 0.5) * (out[t] + xi[t]);
    }
    free(xi);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Newton iterations with the stopping rule of Sec. 5.3: X_0 = M, and         */
/*   variant 0 (matrix sign, eq. "iter"):      X_{k+1} = (X_k + X_k^{-1}) / 2, */
/*   variant 1 (polar factor, eq. "iter2"):    X_{k+1} = (X_k + X_k^{-H}) / 2, */
/* stopping after the first step k with ||X_k - X_{k-1}||_max / ||X_k||_max   */
/* <= eps (max of the entries' moduli), or after kmax steps.  Each inverse is */
/* the right inverse by complex LU.  *steps receives the number of steps.    */
/* ------------------------------------------------------------------------- */
int orc_newton(int n, const zc *m, int variant, double eps, int kmax, zc *out, int *steps)
{
    if (n < 1 || kmax < 0 || (variant != 0 && variant != 1)) return -2;
    size_t nn = (size_t)n * n;
    zc *xi = malloc(sizeof(zc) * nn);
    if (!xi) return -1;
    memcpy(out, m, sizeof(zc) * nn);
    *steps = 0;
    for (int k = 1; k <= kmax; ++k) {
        int info = orc_cplx_lu_inv(n, out, xi, 0);
        if (info) { free(xi); return info; }
        double dmax = 0.0, xmax = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                zc inv = (variant == 1 && ORC_MUTANT != 11) ? conj(xi[IDX(j, i)]) : xi[IDX(i, j)];
                zc nx = 0.5 * (out[IDX(i, j)] + inv);
                double d = abs2(nx - out[IDX(i, j)]), a = abs2(nx);
                if (d > dmax) dmax = d;
                if (a > xmax) xmax = a;
                out[IDX(i, j)] = nx;
            }
        *steps = k;
        if (sqrt(dmax) <= eps * sqrt(xmax)) break;
    }
    free(xi);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Sylvester equation A Y + Y B = C (Sec. 5.4), A p x p, B q x q, C p x q:   */
/* if sign(A) = I_p and sign(B) = I_q, the sign of [[A, -C], [0, -B]] is      */
/* [[I_p, -2Y], [0, -I_q]]; Newton's iteration (variant 0 above) on that      */
/* block matrix, then Y = -1/2 times the top-right block of the limit.        */
/* ------------------------------------------------------------------------- */
int orc_sylvester(int p, int q, const zc *a, const zc *b, const zc *c, double eps, int kmax, zc *y, int *steps)
{
    if (p < 1 || q < 1) return -2;
    const int n = p + q;
    zc *x0 = calloc((size_t)n * n, sizeof(zc)), *xs = malloc(sizeof(zc) * (size_t)n * n);
    if (!x0 || !xs) { free(x0); free(xs); return -1; }
    for (int i = 0; i < p; ++i) {
        for (int j = 0; j < p; ++j) x0[IDX(i, j)] = a[(size_t)i * p + j];
        for (int j = 0; j < q; ++j) x0[IDX(i, p + j)] = -c[(size_t)i * q + j];
    }
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) x0[IDX(p + i, p + j)] = -b[(size_t)i * q + j];
    int info = orc_newton(n, x0, 0, eps, kmax, xs, steps);
    if (info == 0)
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < q; ++j) y[(size_t)i * q + j] = (ORC_MUTANT == 12 ? 0.5 : -0.5) * xs[IDX(i, p + j)];
    free(x0);
    free(xs);
    return info;
}

/* ------------------------------------------------------------------------- */
/* Polar decomposition X = Q P (Sec. 5.5): Q by Newton's iteration variant 1  */
/* above from X_0 = X, then P = Q^H X.                                        */
/* ------------------------------------------------------------------------- */
int orc_polar(int n, const zc *x, double eps, int kmax, zc *q, zc *pm, int *steps)
{
    int info = orc_newton(n, x, 1, eps, kmax, q, steps);
    if (info) return info;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            zc s = 0.0;
            for (int k = 0; k < n; ++k) s += (ORC_MUTANT == 13 ? q[IDX(i, k)] : conj(q[IDX(k, i)])) * x[IDX(k, j)];
            pm[IDX(i, j)] = s;
        }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Algorithm "Linear system with Frobenius inversion" (Sec. 3) for nrhs      */
/* right-hand sides c + i d (n x nrhs, row-major complex):                   */
/* A = P1^T L1 U1; L1 U1 X1 = P1 B; X2 = A + B X1; X2 = P2^T L2 U2;           */
/* L2 U2 [x1, y1] = P2 [c, d]; L1 U1 [x2, y2] = P1 B [y1, x1];               */
/* x = x1 + x2, y = y1 - y2.                                                  */
/* The printed last step reads y = y2 - y1; by eq. (1.1) the imaginary part  */
/* of M^{-1}(c + i d) is S^{-1} d - A^{-1} B S^{-1} c = y1 - y2, which the     */
/* pins confirm.                                                              */
/* ------------------------------------------------------------------------- */

/* Solve L U X = P C for a real n x m right-hand side (row-major, ld m). */
static void dlu_solve_rhs(int n, int m, const double *lu, const int *piv, double *c)
{
    for (int k = 0; k < n; ++k) {
        int p = piv[k];
        if (p != k)
            for (int j = 0; j < m; ++j) { double t = c[(size_t)k * m + j]; c[(size_t)k * m + j] = c[(size_t)p * m + j]; c[(size_t)p * m + j] = t; }
    }
#pragma omp parallel for schedule(static)
    for (int j = 0; j < m; ++j) {
        for (int i = 0; i < n; ++i) {
            double s = c[(size_t)i * m + j];
            for (int k = 0; k < i; ++k) s -= lu[IDX(i, k)] * c[(size_t)k * m + j];
            c[(size_t)i * m + j] = s;
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = c[(size_t)i * m + j];
            for (int k = i + 1; k < n; ++k) s -= lu[IDX(i, k)] * c[(size_t)k * m + j];
            c[(size_t)i * m + j] = s / lu[IDX(i, i)];
        }
    }
}

int orc_frob_solve(int n, int nrhs, const zc *m, const zc *rhs, zc *x)
{
    if (n < 1 || nrhs < 1) return -2;
    size_t nn = (size_t)n * n, nm = (size_t)n * nrhs;
    double *w = malloc(sizeof(double) * (nn * 5 + nm * 4));
    int *piv1 = malloc(sizeof(int) * (size_t)n), *piv2 = malloc(sizeof(int) * (size_t)n);
    if (!w || !piv1 || !piv2) { free(w); free(piv1); free(piv2); return -1; }
    double *A = w, *B = w + nn, *LU1 = w + 2 * nn, *X1 = w + 3 * nn, *X2 = w + 4 * nn;
    double *CD = w + 5 * nn;           /* [c | d], n x 2 nrhs, becomes [x1 | y1] */
    double *T = CD + 2 * nm;           /* B [y1 | x1], becomes [x2 | y2] */
    split_planes(n, m, A, B);
    memcpy(LU1, A, sizeof(double) * nn);
    int info = dgetrf_plain(n, LU1, piv1);                        /* step 1 */
    if (info) goto done;
    memcpy(X1, B, sizeof(double) * nn);
    dlu_solve_cols(n, LU1, piv1, X1);                             /* step 2 */
    dgemm_plain(n, B, X1, A, X2);                                 /* step 3 */
    info = dgetrf_plain(n, X2, piv2);                             /* step 4 */
    if (info) { info += n; goto done; }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < nrhs; ++j) {
            CD[(size_t)i * 2 * nrhs + j] = creal(rhs[(size_t)i * nrhs + j]);
            CD[(size_t)i * 2 * nrhs + nrhs + j] = cimag(rhs[(size_t)i * nrhs + j]);
        }
    dlu_solve_rhs(n, 2 * nrhs, X2, piv2, CD);                      /* step 5 */
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)                                   /* step 6: B [y1, x1] */
        for (int j = 0; j < nrhs; ++j) {
            double sy = 0.0, sx = 0.0;
            for (int k = 0; k < n; ++k) {
                sy += B[IDX(i, k)] * CD[(size_t)k * 2 * nrhs + nrhs + j];
                sx += B[IDX(i, k)] * CD[(size_t)k * 2 * nrhs + j];
            }
            T[(size_t)i * 2 * nrhs + j] = sy;
            T[(size_t)i * 2 * nrhs + nrhs + j] = sx;
        }
    dlu_solve_rhs(n, 2 * nrhs, LU1, piv1, T);
    for (int i = 0; i < n; ++i)                                   /* step 7 */
        for (int j = 0; j < nrhs; ++j) {
            double x1 = CD[(size_t)i * 2 * nrhs + j], y1 = CD[(size_t)i * 2 * nrhs + nrhs + j];
            double x2 = T[(size_t)i * 2 * nrhs + j], y2 = T[(size_t)i * 2 * nrhs + nrhs + j];
            x[(size_t)i * nrhs + j] = (x1 + x2) + I * (ORC_MUTANT == 10 ? y2 - y1 : y1 - y2);
        }
done:
    free(w);
    free(piv1);
    free(piv2);
    return info;
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
