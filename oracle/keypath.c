/*
 * Oracle key path (FP32).  Test infrastructure only; see oracle.h.
 *
 * The tile binning of the rasterizer (Sec. 4: the 3D Gaussian Splatting
 * kernel, reused) turns floating point into integers: a Gaussian is culled or
 * not, covers a rectangle of 16x16 tiles, and is ordered inside each tile by
 * its view-space depth.  Those integers must be identical on both sides, so
 * the quantities that decide them -- depth, screen mean, 2D covariance,
 * radius and rectangle -- are defined here as one fixed FP32 computation:
 * every product-sum is an explicit fmaf chain, division and square root are
 * IEEE (correctly rounded), nothing is contracted (build with
 * -ffp-contract=off) and the only transcendental, exp of the log-scale, is
 * evaluated by orc_exp_f32 below instead of a libm routine.
 *
 * Readings (3DGS conventions the paper inherits without restating):
 *   near plane: culled unless t_z > near (0.2)
 *   Jacobian guard band: t_x/t_z clamped to +-1.3 * (W/2)/f_x inside J only
 *   low-pass dilation: +0.3 px^2 on the diagonal of the 2D covariance
 *   radius: ceil(3 * sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1, mid^2 - det))
 *   rectangle: [floor((mu - r)/16), floor((mu + r + 15)/16)) clamped to the tile grid
 *
 * Tile ellipse (an addition of this implementation, not of the paper): inside
 * its rectangle a Gaussian is binned only to the tiles whose pixel centres can
 * reach alpha >= 1/255.  With Sigma2 = [[a, b], [b, c]] and o its opacity, the
 * pixels where o exp(-q/2) >= 1/255, q = d^T Sigma2^-1 d, form the ellipse
 * q <= 2 ln(255 o).  The key path stores, per Gaussian, a conservative version
 * of that ellipse from which every tile row's span of tiles follows (see
 * orc_row_span in binning.c):
 *   t      = (2 lnu(255 o) + 1/16) (1 + 2^-10),   lnu(x) >= ln(x) (orc_ln_up_f32)
 *   mm     = c t                 (the ellipse's squared half-height)
 *   ystar  = b sqrt(t / a)       (row offset of its right-most point)
 *   s, k   = b / c, det / c^2    (row dy spans dx in s dy +- sqrt(k (mm - dy^2)))
 *   padx/y = 1/4 + 2^-12 (|mu| + 2 r)   (rounding allowance, pixels)
 * The 1/16 and 2^-10 margins absorb the rounding of o, of the conic and of
 * the renderer's exponent, so a tile left out could never have passed the
 * renderer's alpha test: images and gradients are those of rectangle binning.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

/* 2^n for integer n in the normal range, built from its bit pattern (exact). */
static float pow2i(int n)
{
    uint32_t b = (uint32_t)(n + 127) << 23;
    float f;
    memcpy(&f, &b, 4);
    return f;
}

/*
 * exp(x) in FP32 by Cody-Waite argument reduction and a Taylor polynomial:
 *   n = rint(x / ln 2),  r = x - n ln2  (ln2 split into a 16-bit head, so n*head
 *   is exact, and a tail),  e^r = sum_{k<=7} r^k / k!  (|r| <= ln2/2, truncation
 *   error < 6e-9), evaluated in Horner form with fused multiply-adds, then
 *   scaled by 2^n.  Inputs are clamped to [-80, 80] (normal range).
 */
float orc_exp_f32(float x)
{
    const float log2e = 0x1.715476p+0f;
    const float ln2_hi = 0x1.62e4p-1f;
    const float ln2_lo = 0x1.7f7d1cp-20f;
    if (x > 80.f) x = 80.f;
    if (x < -80.f) x = -80.f;
    float n = rintf(x * log2e);
    float r = fmaf(-n, ln2_hi, x);
    r = fmaf(-n, ln2_lo, r);
    float p = 0x1.a01a02p-13f;           /* 1/7! */
    p = fmaf(p, r, 0x1.6c16c2p-10f);     /* 1/6! */
    p = fmaf(p, r, 0x1.111112p-7f);      /* 1/5! */
    p = fmaf(p, r, 0x1.555556p-5f);      /* 1/4! */
    p = fmaf(p, r, 0x1.555556p-3f);      /* 1/3! */
    p = fmaf(p, r, 0x1p-1f);             /* 1/2! */
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    return p * pow2i((int)n);
}

/*
 * Upper bound of ln(x) for normal x > 0, exact to within 0.0141:
 *   x = m 2^e with m in [1, 2) read from the bit pattern (exact), and
 *   ln m <= (m - 1) / sqrt(m)  for m >= 1
 * (the difference has derivative (sqrt(m) - 1)^2 / (2 m^1.5) >= 0 and is 0 at
 * m = 1; at m = 2 it is 1/sqrt(2) - ln 2 = 0.0140).
 */
float orc_ln_up_f32(float x)
{
    uint32_t bits;
    memcpy(&bits, &x, 4);
    const int e = (int)(bits >> 23) - 127;
    const uint32_t mb = (bits & 0x7fffffu) | 0x3f800000u;
    float m;
    memcpy(&m, &mb, 4);
    return (float)e * 0x1.62e430p-1f + (m - 1.0f) / sqrtf(m);
}

static float fclampf(float v, float lo, float hi)
{
    return fminf(fmaxf(v, lo), hi);
}

void orc_keypath(int N, const float* means, const float* log_scales, const float* quats,
                 const float* opacity_raw, const orc_cam* cam, float* depth, float* mean2d, float* cov2d,
                 int32_t* radius, int32_t* rect, int32_t* tiles, float* ell)
{
    const float* V = cam->view;
    const int TX = (cam->W + ORC_TILE - 1) / ORC_TILE;
    const int TY = (cam->H + ORC_TILE - 1) / ORC_TILE;
    const float limx = 1.3f * ((0.5f * (float)cam->W) / cam->fx);
    const float limy = 1.3f * ((0.5f * (float)cam->H) / cam->fy);

    for (int i = 0; i < N; ++i) {
        const float px = means[3 * i], py = means[3 * i + 1], pz = means[3 * i + 2];
        /* view-space position t = R_c p + t_c */
        const float tx = fmaf(V[0], px, fmaf(V[1], py, fmaf(V[2], pz, V[3])));
        const float ty = fmaf(V[4], px, fmaf(V[5], py, fmaf(V[6], pz, V[7])));
        const float tz = fmaf(V[8], px, fmaf(V[9], py, fmaf(V[10], pz, V[11])));
        depth[i] = tz;
        mean2d[2 * i] = mean2d[2 * i + 1] = 0.f;
        cov2d[3 * i] = cov2d[3 * i + 1] = cov2d[3 * i + 2] = 0.f;
        radius[i] = 0;
        rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
        tiles[i] = 0;
        for (int k = 0; k < 8; ++k) ell[8 * i + k] = 0.f;
        if (!(tz > cam->near_z)) continue;

        /* scales and unit quaternion (w, x, y, z) */
        const float s0 = orc_exp_f32(log_scales[3 * i]);
        const float s1 = orc_exp_f32(log_scales[3 * i + 1]);
        const float s2 = orc_exp_f32(log_scales[3 * i + 2]);
        float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
        const float n2 = fmaf(qw, qw, fmaf(qx, qx, fmaf(qy, qy, qz * qz)));
        const float inv = 1.0f / sqrtf(n2);
        qw *= inv; qx *= inv; qy *= inv; qz *= inv;

        const float xx = qx * qx, yy = qy * qy, zz = qz * qz;
        const float xy = qx * qy, xz = qx * qz, yz = qy * qz;
        const float wx = qw * qx, wy = qw * qy, wz = qw * qz;
        float R[3][3];
        R[0][0] = 1.f - 2.f * (yy + zz); R[0][1] = 2.f * (xy - wz);        R[0][2] = 2.f * (xz + wy);
        R[1][0] = 2.f * (xy + wz);        R[1][1] = 1.f - 2.f * (xx + zz); R[1][2] = 2.f * (yz - wx);
        R[2][0] = 2.f * (xz - wy);        R[2][1] = 2.f * (yz + wx);        R[2][2] = 1.f - 2.f * (xx + yy);

        /* M = R diag(s), Sigma = M M^T */
        float M[3][3];
        for (int r = 0; r < 3; ++r) {
            M[r][0] = R[r][0] * s0;
            M[r][1] = R[r][1] * s1;
            M[r][2] = R[r][2] * s2;
        }
        float S[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = r; c < 3; ++c) {
                S[r][c] = fmaf(M[r][0], M[c][0], fmaf(M[r][1], M[c][1], M[r][2] * M[c][2]));
                S[c][r] = S[r][c];
            }

        /* projection Jacobian with guard band */
        const float inv_tz = 1.0f / tz;
        const float xn = tx * inv_tz, yn = ty * inv_tz;
        const float xc = fclampf(xn, -limx, limx);
        const float yc = fclampf(yn, -limy, limy);
        const float J00 = cam->fx * inv_tz;
        const float J02 = -(cam->fx * xc) * inv_tz;
        const float J11 = cam->fy * inv_tz;
        const float J12 = -(cam->fy * yc) * inv_tz;

        /* T = J R_c (2x3) */
        float T0[3], T1[3];
        for (int j = 0; j < 3; ++j) {
            T0[j] = fmaf(J00, V[j], J02 * V[8 + j]);
            T1[j] = fmaf(J11, V[4 + j], J12 * V[8 + j]);
        }
        /* U = T Sigma, cov2d = U T^T + 0.3 I */
        float U0[3], U1[3];
        for (int k = 0; k < 3; ++k) {
            U0[k] = fmaf(T0[0], S[0][k], fmaf(T0[1], S[1][k], T0[2] * S[2][k]));
            U1[k] = fmaf(T1[0], S[0][k], fmaf(T1[1], S[1][k], T1[2] * S[2][k]));
        }
        const float a = fmaf(U0[0], T0[0], fmaf(U0[1], T0[1], U0[2] * T0[2])) + 0.3f;
        const float b = fmaf(U0[0], T1[0], fmaf(U0[1], T1[1], U0[2] * T1[2]));
        const float c = fmaf(U1[0], T1[0], fmaf(U1[1], T1[1], U1[2] * T1[2])) + 0.3f;
        const float det = fmaf(a, c, -(b * b));
        if (!(det > 0.f)) continue;

        const float mx = fmaf(cam->fx, xn, cam->cx);
        const float my = fmaf(cam->fy, yn, cam->cy);
        const float mid = 0.5f * (a + c);
        const float disc = fmaxf(0.1f, fmaf(mid, mid, -det));
        const float lam = mid + sqrtf(disc);
        const float rf = fminf(ceilf(3.0f * sqrtf(lam)), 1048576.0f);

        const int x0 = (int)fclampf(floorf((mx - rf) * 0.0625f), 0.f, (float)TX);
        const int x1 = (int)fclampf(floorf(((mx + rf) + 15.0f) * 0.0625f), 0.f, (float)TX);
        const int y0 = (int)fclampf(floorf((my - rf) * 0.0625f), 0.f, (float)TY);
        const int y1 = (int)fclampf(floorf(((my + rf) + 15.0f) * 0.0625f), 0.f, (float)TY);
        const int nt = (x1 - x0) * (y1 - y0);
        if (nt <= 0) continue;

        mean2d[2 * i] = mx;
        mean2d[2 * i + 1] = my;
        cov2d[3 * i] = a;
        cov2d[3 * i + 1] = b;
        cov2d[3 * i + 2] = c;
        radius[i] = (int32_t)rf;
        rect[4 * i] = x0;
        rect[4 * i + 1] = y0;
        rect[4 * i + 2] = x1;
        rect[4 * i + 3] = y1;
        tiles[i] = nt;

        /* tile ellipse */
        const float o = 1.0f / (1.0f + orc_exp_f32(-opacity_raw[i]));
        const float t = (2.0f * orc_ln_up_f32(255.0f * o) + 0.0625f) * 1.0009765625f;
        float* E = ell + 8 * i;
        E[0] = mx;
        E[1] = my;
        if (t > 0.f) {
            E[2] = b / c;
            E[3] = det / (c * c);
            E[4] = c * t;
            E[5] = b * sqrtf(t / a);
        } else {
            E[4] = -1.0f;   /* alpha < 1/255 everywhere: no tile */
        }
        E[6] = 0.25f + (fabsf(mx) + 2.0f * rf) * 0x1p-12f;
        E[7] = 0.25f + (fabsf(my) + 2.0f * rf) * 0x1p-12f;
    }
}
