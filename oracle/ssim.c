/*
 * Oracle RGB reconstruction loss with D-SSIM (FP64).  Test infrastructure only.
 *
 * Sec. 4 keeps "the same RGB loss" as 3D Gaussian Splatting without restating
 * it; reading: L = (1 - lambda) L1 + lambda (1 - SSIM), lambda = 0.2, with the
 * SSIM of Wang et al. (2004) as 3DGS computes it: per channel, an 11 x 11
 * Gaussian window (sigma 1.5, normalised), zero padding outside the image
 * ("same" size), C1 = 0.01^2, C2 = 0.03^2,
 *   mu_x = G * x, sigma_x^2 = G * x^2 - mu_x^2, sigma_xy = G * (x y) - mu_x mu_y,
 *   S = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)),
 * SSIM = the mean of S over pixels and channels; L1 = mean |x - y| (gradient
 * sign(x - y), 0 at equality).
 * Gradient: S at q depends on x(p) through mu_x(q), sigma_x^2(q), sigma_xy(q),
 *   dS/dmu_x = 2 mu_y n2 / (d1 d2) - 2 mu_x S / d1,  dS/dsigma_x^2 = -S / d2,
 *   dS/dsigma_xy = 2 n1 / (d1 d2)
 * (n1, n2, d1, d2 the four factors above), and the window derivatives give
 *   sum_q dS(q)/dx(p) = (G * A)(p) + 2 x(p) (G * B)(p) + y(p) (G * C)(p),
 *   A = dS/dmu_x - 2 mu_x dS/dsigma_x^2 - mu_y dS/dsigma_xy, B = dS/dsigma_x^2, C = dS/dsigma_xy
 * (G symmetric; A, B, C zero outside the image).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define R 5
static double win[2 * R + 1];

static void window(void)
{
    double s = 0.0;
    for (int k = -R; k <= R; ++k) s += (win[k + R] = exp(-(double)(k * k) / (2.0 * 1.5 * 1.5)));
    for (int k = 0; k <= 2 * R; ++k) win[k] /= s;
}

/* out = G * in over a W x H plane, zero padding; the 2-D window is the outer
 * product of the 1-D one, applied as a plain double sum. */
static void blur(const double* in, double* out, int W, int H)
{
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double s = 0.0;
            for (int a = -R; a <= R; ++a) {
                const int ii = i + a;
                if (ii < 0 || ii >= H) continue;
                for (int b = -R; b <= R; ++b) {
                    const int jj = j + b;
                    if (jj < 0 || jj >= W) continue;
                    s += win[a + R] * win[b + R] * in[(size_t)ii * W + jj];
                }
            }
            out[(size_t)i * W + j] = s;
        }
}

/* img, target [3][H][W]; loss [3] = (L, L1, SSIM); grad [3][H][W] = dL/dimg
 * (nullable); smap [3][H][W] the SSIM map (nullable). */
void orc_rgb_loss(int W, int H, const double* img, const double* target, double lambda, double* loss, double* grad,
                  double* smap)
{
    window();
    const size_t P = (size_t)W * H;
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double* buf = (double*)malloc(sizeof(double) * P * 13);
    double *xx = buf, *yy = buf + P, *xy = buf + 2 * P, *mx = buf + 3 * P, *my = buf + 4 * P, *sxx = buf + 5 * P,
           *syy = buf + 6 * P, *sxy = buf + 7 * P, *A = buf + 8 * P, *B = buf + 9 * P, *Cc = buf + 10 * P,
           *gA = buf + 11 * P, *gB = buf + 12 * P;
    double* gC = (double*)malloc(sizeof(double) * P);
    double ssum = 0.0, l1 = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double* x = img + c * P;
        const double* y = target + c * P;
        for (size_t i = 0; i < P; ++i) {
            xx[i] = x[i] * x[i];
            yy[i] = y[i] * y[i];
            xy[i] = x[i] * y[i];
            l1 += fabs(x[i] - y[i]);
        }
        blur(x, mx, W, H);
        blur(y, my, W, H);
        blur(xx, sxx, W, H);
        blur(yy, syy, W, H);
        blur(xy, sxy, W, H);
        for (size_t i = 0; i < P; ++i) {
            const double vx = sxx[i] - mx[i] * mx[i], vy = syy[i] - my[i] * my[i], cxy = sxy[i] - mx[i] * my[i];
            const double n1 = 2 * mx[i] * my[i] + C1, n2 = 2 * cxy + C2;
            const double d1 = mx[i] * mx[i] + my[i] * my[i] + C1, d2 = vx + vy + C2;
            const double S = n1 * n2 / (d1 * d2);
            ssum += S;
            if (smap) smap[c * P + i] = S;
            const double dmu = 2 * my[i] * n2 / (d1 * d2) - 2 * mx[i] * S / d1;
            const double dvx = -S / d2;
            const double dcxy = 2 * n1 / (d1 * d2);
            A[i] = dmu - 2 * mx[i] * dvx - my[i] * dcxy;
            B[i] = dvx;
            Cc[i] = dcxy;
        }
        if (grad) {
            blur(A, gA, W, H);
            blur(B, gB, W, H);
            blur(Cc, gC, W, H);
            for (size_t i = 0; i < P; ++i) {
                const double dS = gA[i] + 2 * x[i] * gB[i] + y[i] * gC[i];
                const double s1 = x[i] > y[i] ? 1.0 : (x[i] < y[i] ? -1.0 : 0.0);
                grad[c * P + i] = ((1.0 - lambda) * s1 - lambda * dS) / (3.0 * P);
            }
        }
    }
    l1 /= 3.0 * P;
    const double ssim = ssum / (3.0 * P);
    loss[0] = (1.0 - lambda) * l1 + lambda * (1.0 - ssim);
    loss[1] = l1;
    loss[2] = ssim;
    free(gC);
    free(buf);
}
