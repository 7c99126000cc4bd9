/*
 * Oracle adaptive density control (clone / split / prune).  Test
 * infrastructure only.
 *
 * Sec. 4 keeps 3D Gaussian Splatting's adaptive density control without
 * restating it.  Reading (3DGS's published rule, with its constants as
 * parameters):
 *   statistics, per step: acc_i += |dL/dmean2d_i| (pixels), cnt_i += 1 for
 *     every Gaussian with a nonzero screen radius;
 *   decision, per Gaussian: g_i = acc_i / cnt_i (0 if cnt_i = 0);
 *     pruned  if sigmoid(opacity_raw_i) < min_opacity,
 *     else split if g_i >= grad_thresh and max scale > percent_dense * extent,
 *     else clone if g_i >= grad_thresh,
 *     else kept;
 *   output, in this order: every kept or cloned Gaussian (index order), the
 *     clones (index order), the two children of every split Gaussian (index
 *     order).  A clone copies its parent; a child k (k = 0, 1) copies its
 *     parent except mean = mu + R(q) diag(s) n_ik (n_ik the given standard
 *     normal samples, noise[i][k][3]) and log-scale = log-scale - ln(1.6).
 *     Adam moments: carried over for kept Gaussians, zero for clones and
 *     children.
 * Precision: the statistics and the decisions in FP32 with fixed operations
 * (they decide integers; see orc_densify_plan); the child means in FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* kind[i]: 0 pruned, 1 kept, 2 kept + clone, 3 split.  Returns the output count.
 * The three tests in monotone-equivalent forms without transcendental
 * functions, so that every implementation takes the same integer decisions
 * from the same FP32 values (thresholds derived once in double, rounded to FP32):
 *   sigmoid(o) < min_opacity      <=>  o < logit_min  = ln(m / (1 - m))
 *   max scale > percent_dense * E <=>  max log-scale > log_big = ln(percent_dense E)
 *   acc / cnt >= grad_thresh      <=>  cnt > 0 and acc >= fl(grad_thresh * cnt)  (one FP32 product) */
int64_t orc_densify_plan(int n, const float* log_scales, const float* opacity_raw, const float* acc,
                         const int32_t* cnt, float grad_thresh, float log_big, float logit_min, int32_t* kind)
{
    int64_t out = 0;
    for (int i = 0; i < n; ++i) {
        float smax = log_scales[3 * i];
        if (log_scales[3 * i + 1] > smax) smax = log_scales[3 * i + 1];
        if (log_scales[3 * i + 2] > smax) smax = log_scales[3 * i + 2];
        const float lim = grad_thresh * (float)cnt[i];
        const int cand = cnt[i] > 0 && acc[i] >= lim;
        int k;
        if (opacity_raw[i] < logit_min)
            k = 0;
        else if (cand)
            k = smax > log_big ? 3 : 2;
        else
            k = 1;
        kind[i] = k;
        out += k == 0 ? 0 : (k == 1 ? 1 : 2);
    }
    return out;
}

/* Per-step statistics: acc_i += |(g_x, g_y)| = sqrt(g_x g_x + g_y g_y) (FP32,
 * in this order), cnt_i += 1, for every Gaussian with radius_i > 0 (a Gaussian
 * outside the view has radius 0 and no screen-space gradient to count).
 * grad_mean2d: [n][2], the gradient of the loss with respect to each
 * Gaussian's projected mean in pixels. */
void orc_densify_stats(int n, const float* grad_mean2d, const int32_t* radius, float* acc, int32_t* cnt)
{
    for (int i = 0; i < n; ++i) {
        if (radius[i] <= 0) continue;
        const float gx = grad_mean2d[2 * (size_t)i], gy = grad_mean2d[2 * (size_t)i + 1];
        acc[i] += sqrtf(gx * gx + gy * gy);
        cnt[i] += 1;
    }
}

/* Child mean mu + R(q) diag(exp(log_s)) nz, FP64. */
void orc_split_mean(const float* mu, const float* log_s, const float* q, const float* nz, double* out)
{
    const double n = sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] + (double)q[3] * q[3]);
    const double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    const double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                            {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                            {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
    double v[3];
    for (int k = 0; k < 3; ++k) v[k] = exp((double)log_s[k]) * nz[k];
    for (int r = 0; r < 3; ++r) out[r] = mu[r] + R[r][0] * v[0] + R[r][1] * v[1] + R[r][2] * v[2];
}
