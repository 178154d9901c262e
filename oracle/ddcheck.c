/*
 * Compensated (double-double) checks for the MRCQR oracle.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by oracle/mrcqr_oracle.py; never linked
 * into the library.  Sums are Dot2 of Ogita, Rump and Oishi ("Accurate sum
 * and dot product", SIAM J. Sci. Comput. 26(6), 2005): TwoProduct through a
 * fused multiply-add and Knuth's TwoSum, with the error terms accumulated in
 * a second double.  The result is as accurate as if computed in twice the
 * working precision and then rounded once, which is what measuring
 * ||I - Q^T Q|| and ||A - QR|| / ||A|| at the 1e-13 level (Eq. 1, Fig. 1)
 * over m up to 2^22 needs.
 *
 * Build: cc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no -ffast-math:
 * TwoSum must not be reassociated).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

static inline void two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

static inline void two_prod(double a, double b, double *p, double *e) {
    double x = a * b;
    *e = fma(a, b, -x);
    *p = x;
}

/* Dot2 of x and y, length m. */
double dd_dot(int64_t m, const double *x, const double *y) {
    double s = 0.0, c = 0.0;
    for (int64_t k = 0; k < m; ++k) {
        double p, pe, t, te;
        two_prod(x[k], y[k], &p, &pe);
        two_sum(s, p, &t, &te);
        s = t;
        c += te + pe;
    }
    return s + c;
}

/* E = Q^T Q - I (n x n, column-major, ld = n) for Q m x n column-major with
 * leading dimension ldq; every entry is one Dot2 sum that starts from -1 on
 * the diagonal. */
void dd_gram_minus_identity(int64_t m, int64_t n, const double *Q, int64_t ldq, double *E) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t j = 0; j < n; ++j) {
        const double *qj = Q + j * ldq;
        for (int64_t i = 0; i <= j; ++i) {
            const double *qi = Q + i * ldq;
            double s = (i == j) ? -1.0 : 0.0, c = 0.0;
            for (int64_t k = 0; k < m; ++k) {
                double p, pe, t, te;
                two_prod(qi[k], qj[k], &p, &pe);
                two_sum(s, p, &t, &te);
                s = t;
                c += te + pe;
            }
            E[i + j * n] = s + c;
            E[j + i * n] = s + c;
        }
    }
}

/* Res = A - Q R (m x n, column-major, ld = m) for R upper triangular (n x n,
 * ld = ldr); each entry is a Dot2 sum started from a_ij. */
void dd_residual_columns(int64_t m, int64_t n, const double *A, int64_t lda, const double *Q,
                         int64_t ldq, const double *R, int64_t ldr, double *Res) {
#pragma omp parallel
    {
        double *hi = (double *)malloc(sizeof(double) * (size_t)m);
        double *lo = (double *)malloc(sizeof(double) * (size_t)m);
#pragma omp for schedule(dynamic, 1)
        for (int64_t j = 0; j < n; ++j) {
            for (int64_t i = 0; i < m; ++i) {
                hi[i] = A[i + j * lda];
                lo[i] = 0.0;
            }
            for (int64_t k = 0; k <= j; ++k) {
                const double r = -R[k + j * ldr];
                const double *qk = Q + k * ldq;
                for (int64_t i = 0; i < m; ++i) {
                    double p, pe, t, te;
                    two_prod(qk[i], r, &p, &pe);
                    two_sum(hi[i], p, &t, &te);
                    hi[i] = t;
                    lo[i] += te + pe;
                }
            }
            for (int64_t i = 0; i < m; ++i) Res[i + j * m] = hi[i] + lo[i];
        }
        free(hi);
        free(lo);
    }
}
