/*
 * Oracle adaptive density control (clone / split / prune).  Test
 * infrastructure only.
 *
 * Sec. 4 keeps 3D Gaussian Splatting's adaptive density control without
 * restating it.  Reading (3DGS's published rule, with its constants as
 * parameters):
 *   statistics, per step: acc_i += |dL/dmean2d_i| (pixels), cnt_i += 1 and
 *     max_radius_i = max(max_radius_i, radius_i) for every Gaussian with a
 *     nonzero screen radius;
 *   decision, per Gaussian: g_i = acc_i / cnt_i (0 if cnt_i = 0);
 *     pruned  if sigmoid(opacity_raw_i) < min_opacity, or (when enabled) its
 *             largest screen radius exceeds max_screen pixels or its largest
 *             scale exceeds world_frac * extent (3DGS removes Gaussians too
 *             large in view space and in world space),
 *     else split if g_i >= grad_thresh and max scale > percent_dense * extent,
 *     else clone if g_i >= grad_thresh,
 *     else kept;
 *   output, in this order: every kept or cloned Gaussian (index order), the
 *     clones (index order), the two children of every split Gaussian (index
 *     order).  A clone copies its parent; a child k (k = 0, 1) copies its
 *     parent except mean = mu + R(q) diag(s) n_ik (n_ik the given standard
 *     normal samples, noise[i][k][3]) and log-scale = log-scale - ln(1.6).
 *     Adam moments: carried over for kept Gaussians, zero for clones and
 *     children;
 *   opacity reset, every few thousand steps: opacity = min(opacity,
 *     max_opacity) (3DGS: 0.01), with the opacity's Adam moments zeroed.
 * Precision: the statistics and the decisions in FP32 with fixed operations
 * (they decide integers; see orc_densify_plan); the child means in FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* kind[i]: 0 pruned, 1 kept, 2 kept + clone, 3 split.  Returns the output count.
 * The tests in monotone-equivalent forms without transcendental functions, so
 * that every implementation takes the same integer decisions from the same FP32
 * values (thresholds derived once in double, rounded to FP32):
 *   sigmoid(o) < min_opacity          <=>  o < logit_min  = ln(m / (1 - m))
 *   max scale > percent_dense * E     <=>  max log-scale > log_big = ln(percent_dense E)
 *   max scale > world_frac * E        <=>  max log-scale > log_world = ln(world_frac E)
 *   acc / cnt >= grad_thresh          <=>  cnt > 0 and acc >= fl(grad_thresh * cnt)  (one FP32 product)
 * Pruning also removes, when enabled, the Gaussians too large on screen (largest
 * screen radius since the statistics were reset > max_screen, pixels; max_radius
 * may be NULL when max_screen <= 0) or in the world (log_world; +inf = off).  A
 * pruned Gaussian is neither cloned nor split. */
int64_t orc_densify_plan(int n, const float* log_scales, const float* opacity_raw, const float* acc,
                         const int32_t* cnt, const int32_t* max_radius, float grad_thresh, float log_big,
                         float logit_min, float max_screen, float log_world, int32_t* kind)
{
    int64_t out = 0;
    for (int i = 0; i < n; ++i) {
        float smax = log_scales[3 * i];
        if (log_scales[3 * i + 1] > smax) smax = log_scales[3 * i + 1];
        if (log_scales[3 * i + 2] > smax) smax = log_scales[3 * i + 2];
        const float lim = grad_thresh * (float)cnt[i];
        const int cand = cnt[i] > 0 && acc[i] >= lim;
        const int big_screen = max_screen > 0.0f && (float)max_radius[i] > max_screen;
        const int big_world = smax > log_world;
        int k;
        if (opacity_raw[i] < logit_min || big_screen || big_world)
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

/* 3DGS's periodic opacity reset: every opacity above max_opacity is lowered to
 * it, i.e. opacity_raw = min(opacity_raw, logit_max) with logit_max =
 * fl(ln(max_opacity / (1 - max_opacity))), and the opacity's Adam moments restart
 * from zero. */
void orc_opacity_reset(int n, float* opacity_raw, float* m, float* v, float logit_max)
{
    for (int i = 0; i < n; ++i) {
        if (opacity_raw[i] > logit_max) opacity_raw[i] = logit_max;
        m[i] = 0.0f;
        v[i] = 0.0f;
    }
}

/* Per-step statistics: acc_i += |(g_x, g_y)| = sqrt(g_x g_x + g_y g_y) (FP32,
 * in this order), cnt_i += 1, and max_radius_i = max(max_radius_i, radius_i)
 * (max_radius may be NULL), for every Gaussian with radius_i > 0 (a Gaussian
 * outside the view has radius 0 and no screen-space gradient to count).
 * grad_mean2d: [n][2], the gradient of the loss with respect to each
 * Gaussian's projected mean in pixels. */
void orc_densify_stats(int n, const float* grad_mean2d, const int32_t* radius, float* acc, int32_t* cnt,
                       int32_t* max_radius)
{
    for (int i = 0; i < n; ++i) {
        if (radius[i] <= 0) continue;
        const float gx = grad_mean2d[2 * (size_t)i], gy = grad_mean2d[2 * (size_t)i + 1];
        acc[i] += sqrtf(gx * gx + gy * gy);
        cnt[i] += 1;
        if (max_radius && radius[i] > max_radius[i]) max_radius[i] = radius[i];
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
