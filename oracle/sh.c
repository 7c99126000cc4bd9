/*
 * Oracle real spherical harmonics (FP64).  Test infrastructure only.
 *
 * The view-dependent colour c of a Gaussian (Eq. 1, the "color c" attribute;
 * the paper reuses 3DGS, Sec. 4) is sum_lm Y_lm(dir) k_lm + 0.5, clamped at 0,
 * over real SH of degree <= 3.  The basis is written generically from its
 * textbook definition instead of expanded polynomials:
 *
 *   P_l^m(z) = (-1)^m (1 - z^2)^{m/2} d^m P_l / dz^m      (Condon-Shortley phase)
 *   K_l^m    = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
 *   Y_l0     = K_l^0 P_l(z)
 *   Y_lm     = sqrt2 K_l^m P_l^m(cos th) cos(m ph)      m > 0
 *   Y_l,-m   = sqrt2 K_l^m P_l^m(cos th) sin(m ph)      m > 0
 *
 * On the unit sphere (1-z^2)^{m/2} cos(m ph) = Re (x + i y)^m and likewise Im for
 * sin, so each Y is the polynomial  c_lm * D_lm(z) * Re|Im (x + i y)^m  with
 * D_lm = d^m P_l / dz^m.  Its Cartesian gradient (used by the backward pass,
 * which projects it onto the sphere's tangent plane) follows from
 * d/dz D_lm = D_l,m+1,  d/dx (x+iy)^m = m (x+iy)^{m-1},  d/dy (x+iy)^m = i m (x+iy)^{m-1}.
 *
 * Coefficient order: k = l^2 + l + m for m = -l..l (reading; any fixed order
 * works as long as both sides use it).
 */
#include <math.h>
#include "oracle.h"

#define LMAX 3

int orc_sh_count(int deg) { return (deg + 1) * (deg + 1); }

/* Legendre polynomial coefficients leg[l][p] (coefficient of z^p), Bonnet recurrence. */
static void legendre_coeffs(double leg[LMAX + 2][LMAX + 2])
{
    for (int l = 0; l < LMAX + 2; ++l)
        for (int p = 0; p < LMAX + 2; ++p) leg[l][p] = 0.0;
    leg[0][0] = 1.0;
    leg[1][1] = 1.0;
    for (int n = 1; n + 1 <= LMAX; ++n)
        for (int p = 0; p <= n + 1; ++p) {
            double a = (p >= 1) ? (2.0 * n + 1.0) * leg[n][p - 1] : 0.0;
            double b = n * leg[n - 1][p];
            leg[n + 1][p] = (a - b) / (n + 1.0);
        }
}

/* m-th derivative of P_l evaluated at z. */
static double dlegendre(const double leg[LMAX + 2][LMAX + 2], int l, int m, double z)
{
    if (m > l) return 0.0;
    double s = 0.0, zp = 1.0;
    for (int p = m; p <= l; ++p) {
        double fall = 1.0;                      /* p (p-1) ... (p-m+1) */
        for (int j = 0; j < m; ++j) fall *= (double)(p - j);
        s += leg[l][p] * fall * zp;
        zp *= z;
    }
    return s;
}

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* (x + i y)^m as (re, im) */
static void xy_pow(double x, double y, int m, double* re, double* im)
{
    double r = 1.0, i = 0.0;
    for (int k = 0; k < m; ++k) {
        double nr = r * x - i * y;
        double ni = r * y + i * x;
        r = nr;
        i = ni;
    }
    *re = r;
    *im = i;
}

void orc_sh_basis(int deg, const double dir[3], double* Y, double* dY)
{
    double leg[LMAX + 2][LMAX + 2];
    legendre_coeffs(leg);
    const double x = dir[0], y = dir[1], z = dir[2];
    for (int l = 0; l <= deg; ++l) {
        for (int m = 0; m <= l; ++m) {
            const double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m));
            const double sgn = (m % 2) ? -1.0 : 1.0;
            const double c = (m == 0) ? K : sqrt(2.0) * K * sgn;
            const double D = dlegendre(leg, l, m, z);
            const double Dz = dlegendre(leg, l, m + 1, z);
            double re, im, re1 = 0.0, im1 = 0.0;
            xy_pow(x, y, m, &re, &im);
            if (m > 0) xy_pow(x, y, m - 1, &re1, &im1);
            /* cosine-type (m >= 0): Re (x+iy)^m */
            const int kc = l * l + l + m;
            Y[kc] = c * D * re;
            if (dY) {
                dY[3 * kc + 0] = c * D * m * re1;
                dY[3 * kc + 1] = c * D * (-m * im1);
                dY[3 * kc + 2] = c * Dz * re;
            }
            if (m > 0) {
                const int ks = l * l + l - m;
                Y[ks] = c * D * im;
                if (dY) {
                    dY[3 * ks + 0] = c * D * m * im1;
                    dY[3 * ks + 1] = c * D * m * re1;
                    dY[3 * ks + 2] = c * Dz * im;
                }
            }
        }
    }
}
