/*
 * Plain FP64 banded LU factorisation, banded triangular solves and banded
 * matrix-vector products.  TEST INFRASTRUCTURE ONLY: this file is part of the
 * CPU oracle.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it; the product library never does.
 *
 * These are the textbook loops the paper relies on for the per-partition
 * "D-stage" (paper section 2.1, "SPIKE partitioning": A = D S with D holding the
 * diagonal blocks A_i, which are factorised and solved independently; section
 * 3.3 states that each A_i is factorised by a direct solver).  Nothing here is
 * blocked, fused or reordered.
 *
 * Storage (LAPACK band convention, with kl = ku = k):
 *   input band  ab[(k + i - j) * ld + j]      = A[i][j],  |i - j| <= k,  2k+1 rows
 *   unpivoted LU: same layout, U on rows 0..k (diagonal at row k),
 *                 L multipliers on rows k+1..2k (unit diagonal implied)
 *   pivoted LU:   3k+1 rows, A[i][j] at row 2k + i - j; U gains k more
 *                 superdiagonals from row interchanges (rows 0..2k), L on
 *                 rows 2k+1..3k, ipiv[j] = row swapped with row j (0-based).
 * Right-hand sides are column-major with leading dimension ldb.
 */
#include <math.h>
#include <stdint.h>

#define NP(i, j) ab[(int64_t)(k + (i) - (j)) * ld + (j)]      /* unpivoted layout */
#define PV(i, j) ab[(int64_t)(2 * k + (i) - (j)) * ld + (j)]  /* pivoted layout   */

static int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }

/* Doolittle LU without pivoting, in place.  Returns 0, or j+1 when the pivot
 * of column j is zero or not finite. */
int oracle_band_lu_nopiv(int64_t n, int32_t k, double *ab, int64_t ld)
{
    for (int64_t j = 0; j < n; ++j) {
        double piv = NP(j, j);
        if (piv == 0.0 || !isfinite(piv)) return (int)(j + 1);
        int64_t last = imin(n - 1, j + k);
        for (int64_t i = j + 1; i <= last; ++i) {
            double l = NP(i, j) / piv;
            NP(i, j) = l;
            for (int64_t c = j + 1; c <= last; ++c) NP(i, c) -= l * NP(j, c);
        }
    }
    return 0;
}

/* LU with partial pivoting restricted to the band (the gbtf2 scheme): the pivot
 * of column j is the entry of largest magnitude among rows j..j+k, the lowest
 * row winning ties; rows j and ipiv[j] are swapped over columns j..j+2k.
 * ab must hold 3k+1 rows with the band on rows k..3k and zeros on rows 0..k-1. */
int oracle_band_lu_piv(int64_t n, int32_t k, double *ab, int64_t ld, int32_t *ipiv)
{
    for (int64_t j = 0; j < n; ++j) {
        int64_t last = imin(n - 1, j + k);
        int64_t best = j;
        for (int64_t i = j + 1; i <= last; ++i)
            if (fabs(PV(i, j)) > fabs(PV(best, j))) best = i;
        ipiv[j] = (int32_t)best;
        if (PV(best, j) == 0.0 || !isfinite(PV(best, j))) return (int)(j + 1);
        int64_t cend = imin(n - 1, j + 2 * (int64_t)k);
        if (best != j) {
            for (int64_t c = j; c <= cend; ++c) {
                double t = PV(j, c);
                PV(j, c) = PV(best, c);
                PV(best, c) = t;
            }
        }
        double piv = PV(j, j);
        for (int64_t i = j + 1; i <= last; ++i) {
            double l = PV(i, j) / piv;
            PV(i, j) = l;
            for (int64_t c = j + 1; c <= cend; ++c) PV(i, c) -= l * PV(j, c);
        }
    }
    return 0;
}

/* Solve A X = B (trans = 0) or A^T X = B (trans = 1) with the unpivoted factors;
 * B is overwritten with X. */
void oracle_band_solve_nopiv(int64_t n, int32_t k, const double *ab, int64_t ld,
                             double *b, int64_t ldb, int32_t nrhs, int32_t trans)
{
    for (int32_t q = 0; q < nrhs; ++q) {
        double *x = b + (int64_t)q * ldb;
        if (!trans) {
            for (int64_t j = 0; j < n; ++j)                     /* L y = b */
                for (int64_t i = j + 1; i <= imin(n - 1, j + k); ++i) x[i] -= NP(i, j) * x[j];
            for (int64_t j = n - 1; j >= 0; --j) {              /* U x = y */
                x[j] /= NP(j, j);
                for (int64_t i = imax(0, j - k); i < j; ++i) x[i] -= NP(i, j) * x[j];
            }
        } else {
            for (int64_t j = 0; j < n; ++j) {                   /* U^T y = b */
                double s = x[j];
                for (int64_t i = imax(0, j - k); i < j; ++i) s -= NP(i, j) * x[i];
                x[j] = s / NP(j, j);
            }
            for (int64_t j = n - 1; j >= 0; --j) {              /* L^T x = y */
                double s = x[j];
                for (int64_t i = j + 1; i <= imin(n - 1, j + k); ++i) s -= NP(i, j) * x[i];
                x[j] = s;
            }
        }
    }
}

/* Same with the pivoted factors (L is kept in product form, as gbtf2 leaves it). */
void oracle_band_solve_piv(int64_t n, int32_t k, const double *ab, int64_t ld,
                           const int32_t *ipiv, double *b, int64_t ldb, int32_t nrhs,
                           int32_t trans)
{
    for (int32_t q = 0; q < nrhs; ++q) {
        double *x = b + (int64_t)q * ldb;
        if (!trans) {
            for (int64_t j = 0; j < n; ++j) {
                int64_t pj = ipiv[j];
                if (pj != j) { double t = x[j]; x[j] = x[pj]; x[pj] = t; }
                for (int64_t i = j + 1; i <= imin(n - 1, j + k); ++i) x[i] -= PV(i, j) * x[j];
            }
            for (int64_t j = n - 1; j >= 0; --j) {
                x[j] /= PV(j, j);
                for (int64_t i = imax(0, j - 2 * (int64_t)k); i < j; ++i) x[i] -= PV(i, j) * x[j];
            }
        } else {
            for (int64_t j = 0; j < n; ++j) {
                double s = x[j];
                for (int64_t i = imax(0, j - 2 * (int64_t)k); i < j; ++i) s -= PV(i, j) * x[i];
                x[j] = s / PV(j, j);
            }
            for (int64_t j = n - 1; j >= 0; --j) {
                double s = x[j];
                for (int64_t i = j + 1; i <= imin(n - 1, j + k); ++i) s -= PV(i, j) * x[i];
                x[j] = s;
                int64_t pj = ipiv[j];
                if (pj != j) { double t = x[j]; x[j] = x[pj]; x[pj] = t; }
            }
        }
    }
}

/* Y = A X (trans = 0) or Y = A^T X (trans = 1) from the original band. */
void oracle_band_matvec(int64_t n, int32_t k, const double *ab, int64_t ld,
                        const double *xin, int64_t ldx, double *y, int64_t ldy,
                        int32_t nrhs, int32_t trans)
{
    for (int32_t q = 0; q < nrhs; ++q) {
        const double *x = xin + (int64_t)q * ldx;
        double *out = y + (int64_t)q * ldy;
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int64_t j = imax(0, i - k); j <= imin(n - 1, i + k); ++j)
                s += (trans ? NP(j, i) : NP(i, j)) * x[j];
            out[i] = s;
        }
    }
}
