/*
 * Oracle front-to-back compositing of RGB, semantic feature and uncertainty,
 * and its adjoint (FP64).  Test infrastructure only; see oracle.h.
 *
 * Per pixel, over the depth-ordered Gaussians of its tile (Eq. 1 for colour,
 * R_s of Sec. 3.4.1 for the 8-dim feature s_G, R_u of Sec. 3.4.2 for u):
 *   d = mean2d - (px, py)
 *   power = -1/2 (A dx^2 + C dy^2) - B dx dy          conic (A, B, C)
 *   skip if power > 0
 *   alpha = min(0.99, o exp(power));  skip if alpha < 1/255
 *   stop (Gaussian not blended) once T (1 - alpha) < 1e-4
 *   out += f alpha T for the 12 channels, T <- T (1 - alpha)
 *   rgb += T_final bg  (feature and uncertainty backgrounds are 0)
 * Readings: the 0.99 clamp, the 1/255 skip and the 1e-4 stop are the 3DGS
 * constants the paper inherits; n_contrib = 1 + the list position (inside
 * the tile's range) of the last blended Gaussian, 0 if none.
 *
 * flip[px] marks pixels where one of those thresholds is within a hair of
 * deciding differently (|o G - 1/255| < 1e-6, |o G - 0.99| < 1e-6,
 * |T (1 - alpha) - 1e-4| < 2e-8): FP32 and FP64 may legitimately disagree
 * there, so comparisons exclude them.
 *
 * Backward: the exact adjoint, walking each pixel's blended list from the
 * back with the running "colour behind" acc:
 *   dL/df_i   = alpha_i T_i dL/dC
 *   dL/dalpha_i = sum_ch (f_i - acc_i) T_i dL/dC_ch - T_final/(1 - alpha_i) sum_rgb bg dL/dC
 *   acc <- alpha_i f_i + (1 - alpha_i) acc
 * then through alpha = o G (zero when clamped at 0.99) to o, the conic and
 * the screen mean.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

typedef struct {
    uint32_t g;
    double alpha, T, G, dx, dy;
    int clamped;
} contrib;

/* Front-to-back walk of one pixel; returns the number of blended Gaussians. */
static int walk_pixel(const uint32_t* vals, uint32_t start, uint32_t end, double px, double py,
                      const double* mean2d, const double* conic, const double* opacity,
                      contrib* list, double* T_out, int32_t* ncontrib, uint8_t* flip)
{
    double T = 1.0;
    int n = 0;
    int32_t last = 0;
    uint8_t fl = 0;
    for (uint32_t k = start; k < end; ++k) {
        const uint32_t g = vals[k];
        const double dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
        const double A = conic[3 * g], B = conic[3 * g + 1], C = conic[3 * g + 2];
        const double power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy;
        if (power > 0) continue;
        const double G = exp(power);
        const double a0 = opacity[g] * G;
        if (fabs(a0 - 1.0 / 255.0) < 1e-6 || fabs(a0 - 0.99) < 1e-6) fl = 1;
        const int clamped = a0 >= 0.99;
        const double alpha = clamped ? 0.99 : a0;
        if (alpha < 1.0 / 255.0) continue;
        const double test = T * (1.0 - alpha);
        if (fabs(test - 1e-4) < 2e-8) fl = 1;
        if (test < 1e-4) break;
        list[n].g = g;
        list[n].alpha = alpha;
        list[n].T = T;
        list[n].G = G;
        list[n].dx = dx;
        list[n].dy = dy;
        list[n].clamped = clamped;
        ++n;
        T = test;
        last = (int32_t)(k - start + 1);
    }
    *T_out = T;
    *ncontrib = last;
    *flip = fl;
    return n;
}

static void channels(uint32_t g, const double* rgb, const float* feat, const float* unc, double f[ORC_NCH])
{
    for (int c = 0; c < 3; ++c) f[c] = rgb[3 * g + c];
    for (int c = 0; c < ORC_DFEAT; ++c) f[3 + c] = feat[(size_t)ORC_DFEAT * g + c];
    f[3 + ORC_DFEAT] = unc[g];
}

static uint32_t max_range(const uint32_t* ranges, int ntiles)
{
    uint32_t m = 0;
    for (int t = 0; t < ntiles; ++t)
        if (ranges[2 * t + 1] - ranges[2 * t] > m) m = ranges[2 * t + 1] - ranges[2 * t];
    return m;
}

void orc_render(const orc_cam* cam, int N, const uint32_t* vals, const uint32_t* ranges,
                const double* mean2d, const double* conic, const double* opacity, const double* rgb,
                const float* feat, const float* unc, int x0, int y0, int x1, int y1,
                double* out_rgb, double* out_feat, double* out_unc, double* T_final,
                int32_t* n_contrib, uint8_t* flip)
{
    (void)N;
    const int TX = (cam->W + ORC_TILE - 1) / ORC_TILE;
    const int TY = (cam->H + ORC_TILE - 1) / ORC_TILE;
    const int ww = x1 - x0, wh = y1 - y0;
    const size_t P = (size_t)ww * wh;
    const uint32_t lmax = max_range(ranges, TX * TY);
#pragma omp parallel
    {
        contrib* list = (contrib*)malloc(sizeof(contrib) * (lmax + 1));
#pragma omp for schedule(dynamic, 16)
        for (int y = y0; y < y1; ++y)
            for (int x = x0; x < x1; ++x) {
                const size_t o = (size_t)(y - y0) * ww + (x - x0);
                const int t = (y / ORC_TILE) * TX + (x / ORC_TILE);
                double T;
                const int n = walk_pixel(vals, ranges[2 * t], ranges[2 * t + 1], x, y, mean2d, conic, opacity,
                                         list, &T, &n_contrib[o], &flip[o]);
                double acc[ORC_NCH] = {0};
                for (int i = 0; i < n; ++i) {
                    double f[ORC_NCH];
                    channels(list[i].g, rgb, feat, unc, f);
                    for (int c = 0; c < ORC_NCH; ++c) acc[c] += f[c] * list[i].alpha * list[i].T;
                }
                for (int c = 0; c < 3; ++c) out_rgb[c * P + o] = acc[c] + T * cam->bg[c];
                for (int c = 0; c < ORC_DFEAT; ++c) out_feat[c * P + o] = acc[3 + c];
                out_unc[o] = acc[3 + ORC_DFEAT];
                T_final[o] = T;
            }
        free(list);
    }
}

void orc_render_bwd(const orc_cam* cam, int N, const uint32_t* vals, const uint32_t* ranges,
                    const double* mean2d, const double* conic, const double* opacity, const double* rgb,
                    const float* feat, const float* unc, int x0, int y0, int x1, int y1,
                    const double* dL_drgb, const double* dL_dfeat, const double* dL_dunc,
                    double* d_mean2d, double* d_conic, double* d_opacity, double* d_rgb,
                    double* d_feat, double* d_unc)
{
    const int TX = (cam->W + ORC_TILE - 1) / ORC_TILE;
    const int TY = (cam->H + ORC_TILE - 1) / ORC_TILE;
    const int ww = x1 - x0;
    const size_t P = (size_t)ww * (y1 - y0);
    memset(d_mean2d, 0, sizeof(double) * 2 * N);
    memset(d_conic, 0, sizeof(double) * 3 * N);
    memset(d_opacity, 0, sizeof(double) * N);
    memset(d_rgb, 0, sizeof(double) * 3 * N);
    memset(d_feat, 0, sizeof(double) * ORC_DFEAT * N);
    memset(d_unc, 0, sizeof(double) * N);
    contrib* list = (contrib*)malloc(sizeof(contrib) * (max_range(ranges, TX * TY) + 1));
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            const size_t o = (size_t)(y - y0) * ww + (x - x0);
            const int t = (y / ORC_TILE) * TX + (x / ORC_TILE);
            double Tf;
            int32_t nc;
            uint8_t fl;
            const int n = walk_pixel(vals, ranges[2 * t], ranges[2 * t + 1], x, y, mean2d, conic, opacity,
                                     list, &Tf, &nc, &fl);
            double dC[ORC_NCH];
            for (int c = 0; c < 3; ++c) dC[c] = dL_drgb[c * P + o];
            for (int c = 0; c < ORC_DFEAT; ++c) dC[3 + c] = dL_dfeat[c * P + o];
            dC[3 + ORC_DFEAT] = dL_dunc[o];
            double bgdot = 0;
            for (int c = 0; c < 3; ++c) bgdot += cam->bg[c] * dC[c];
            double acc[ORC_NCH] = {0};
            for (int i = n - 1; i >= 0; --i) {
                const contrib* e = &list[i];
                const uint32_t g = e->g;
                double f[ORC_NCH];
                channels(g, rgb, feat, unc, f);
                double dalpha = 0;
                for (int c = 0; c < ORC_NCH; ++c) {
                    const double w = e->alpha * e->T * dC[c];
                    if (c < 3) d_rgb[3 * g + c] += w;
                    else if (c < 3 + ORC_DFEAT) d_feat[(size_t)ORC_DFEAT * g + (c - 3)] += w;
                    else d_unc[g] += w;
                    dalpha += (f[c] - acc[c]) * e->T * dC[c];
                    acc[c] = e->alpha * f[c] + (1 - e->alpha) * acc[c];
                }
                dalpha -= Tf / (1 - e->alpha) * bgdot;
                if (e->clamped) continue;
                const double A = conic[3 * g], B = conic[3 * g + 1], C = conic[3 * g + 2];
                d_opacity[g] += dalpha * e->G;
                const double dpow = dalpha * e->alpha;
                d_conic[3 * g] += dpow * (-0.5 * e->dx * e->dx);
                d_conic[3 * g + 1] += dpow * (-e->dx * e->dy);
                d_conic[3 * g + 2] += dpow * (-0.5 * e->dy * e->dy);
                d_mean2d[2 * g] += dpow * (-A * e->dx - B * e->dy);
                d_mean2d[2 * g + 1] += dpow * (-C * e->dy - B * e->dx);
            }
        }
    free(list);
}
