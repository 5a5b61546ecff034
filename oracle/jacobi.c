/*
 * One-sided (Hestenes) Jacobi SVD, plain C, FP64, single thread.
 * Test infrastructure only: the CPU oracle's own SVD for the compression
 * step of App. B (Schmidt spectrum of each bond of |rho>>).
 *
 * oracle_jacobi_rows(W, c, L, Z, tol, max_sweeps):
 *   W   c x L row-major; its rows are rotated in place (from the left) until
 *       every pair of rows is orthogonal to |w_p.w_q| <= tol*|w_p||w_q|.
 *       On exit row j = s_j * (unit vector).
 *   Z   optional c x c row-major matrix rotated alongside (NULL to skip).
 *   Returns the number of sweeps used, or -1 if max_sweeps was reached.
 * Ordering: cyclic by rows, (0,1), (0,2), ..., (c-2,c-1).  The three inner
 * products are recomputed for every pair.
 * Numerical zero: a row whose norm is at most DBL_EPSILON * ||W||_F (its
 * direction is rounding noise) is set to exactly zero and never rotated;
 * without this, rows of a rank-deficient W shrink by ~eps per sweep forever.
 */
#include <float.h>
#include <math.h>
#include <stddef.h>

static double dot(const double *a, const double *b, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

int oracle_jacobi_rows(double *W, int c, int L, double *Z, double tol, int max_sweeps) {
    double fro2 = 0.0;
    for (int p = 0; p < c; ++p) fro2 += dot(W + (size_t)p * L, W + (size_t)p * L, L);
    const double floor2 = DBL_EPSILON * DBL_EPSILON * fro2;
    for (int sweep = 1; sweep <= max_sweeps; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < c - 1; ++p) {
            for (int q = p + 1; q < c; ++q) {
                double *wp = W + (size_t)p * L, *wq = W + (size_t)q * L;
                double a = dot(wp, wp, L), b = dot(wq, wq, L), g = dot(wp, wq, L);
                if (a <= floor2 || b <= floor2) {
                    if (a <= floor2) for (int i = 0; i < L; ++i) wp[i] = 0.0;
                    if (b <= floor2) for (int i = 0; i < L; ++i) wq[i] = 0.0;
                    continue;
                }
                if (g == 0.0 || fabs(g) <= tol * sqrt(a) * sqrt(b)) continue;
                rotated = 1;
                double zeta = (b - a) / (2.0 * g);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
                double cs = 1.0 / sqrt(1.0 + t * t);
                double sn = cs * t;
                for (int i = 0; i < L; ++i) {
                    double x = wp[i], y = wq[i];
                    wp[i] = cs * x - sn * y;
                    wq[i] = sn * x + cs * y;
                }
                if (Z) {
                    double *zp = Z + (size_t)p * c, *zq = Z + (size_t)q * c;
                    for (int i = 0; i < c; ++i) {
                        double x = zp[i], y = zq[i];
                        zp[i] = cs * x - sn * y;
                        zq[i] = sn * x + cs * y;
                    }
                }
            }
        }
        if (!rotated) return sweep;
    }
    return -1;
}
