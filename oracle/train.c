/*
 * Oracle RGB L1 loss and Adam step (FP64).  Test infrastructure only.
 *
 * RGB loss: Sec. 4 keeps "the same RGB loss following 3D Gaussian
 * Splatting"; reading: the L1 term only, L = mean |img - target| over all
 * channels and pixels, dL/dimg = sign(img - target) / n (sign(0) = 0).
 *
 * Adam (Sec. 4: lr 1e-3, betas (0.9, 0.999); epsilon is not stated, reading
 * 1e-8; no weight decay):
 *   m <- b1 m + (1-b1) g,   v <- b2 v + (1-b2) g^2
 *   p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
 */
#include <math.h>
#include "oracle.h"

double orc_l1(int64_t n, const double* img, const float* target, double* grad)
{
    double s = 0;
    for (int64_t i = 0; i < n; ++i) {
        const double r = img[i] - (double)target[i];
        s += fabs(r);
        grad[i] = (r > 0 ? 1.0 : (r < 0 ? -1.0 : 0.0)) / (double)n;
    }
    return s / (double)n;
}

void orc_adam(int64_t n, double* param, const double* grad, double* m, double* v, int step,
              double lr, double b1, double b2, double eps)
{
    const double c1 = 1.0 - pow(b1, step);
    const double c2 = 1.0 - pow(b2, step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1 - b1) * grad[i];
        v[i] = b2 * v[i] + (1 - b2) * grad[i] * grad[i];
        param[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
