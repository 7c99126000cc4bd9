/*
 * Oracle projection of 3D Gaussians to screen space, and its adjoint (FP64).
 * Test infrastructure only; see oracle.h.
 *
 * Forward (Eq. 1: the attributes p, Sigma, c, alpha of each Gaussian, Sec. 3.1):
 *   s = exp(log_s), q = q_raw / |q_raw|, R = R(q), Sigma = R S S^T R^T
 *   t = R_c p + t_c                                     view space
 *   J = [[fx/tz, 0, -fx xc/tz], [0, fy/tz, -fy yc/tz]]  xc, yc = clamped t_x/t_z, t_y/t_z
 *   Sigma2 = J R_c Sigma R_c^T J^T + 0.3 I = [[a, b], [b, c]]
 *   conic = Sigma2^{-1} = (c, -b, a) / (ac - b^2)
 *   mean2d = (fx t_x/t_z + cx, fy t_y/t_z + cy), depth = t_z
 *   opacity = sigmoid(opacity_raw)
 *   rgb = max(0, sum_k Y_k(dir) sh_k + 0.5), dir = (p - campos)/|p - campos|
 * A Gaussian is visible iff the FP32 key path gave it at least one tile; the
 * others get zeros here and zero gradients below.
 *
 * Backward: the exact adjoint of every step above (branch taken at the
 * guard-band clamp and the colour clamp), written with explicit matrices.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

typedef struct {
    double p[3], t[3], s[3], q[3 + 1], qnorm, R[3][3], M[3][3], Sig[3][3];
    double Vr[3][3], J[2][3], T[2][3], a, b, c, det, conic[3], xn, yn, xc, yc;
    int clamped_x, clamped_y;
    double o, dir[3], vlen;
} geom;

static void quat_rot(const double q[4], double R[3][3])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* dR[i][j][k] = d R_ij / d q_k, q = (w, x, y, z) */
static void quat_rot_jac(const double q[4], double dR[3][3][4])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    memset(dR, 0, sizeof(double) * 36);
    dR[0][0][2] = -4 * y; dR[0][0][3] = -4 * z;
    dR[0][1][0] = -2 * z; dR[0][1][1] = 2 * y; dR[0][1][2] = 2 * x; dR[0][1][3] = -2 * w;
    dR[0][2][0] = 2 * y;  dR[0][2][1] = 2 * z; dR[0][2][2] = 2 * w; dR[0][2][3] = 2 * x;
    dR[1][0][0] = 2 * z;  dR[1][0][1] = 2 * y; dR[1][0][2] = 2 * x; dR[1][0][3] = 2 * w;
    dR[1][1][1] = -4 * x; dR[1][1][3] = -4 * z;
    dR[1][2][0] = -2 * x; dR[1][2][1] = -2 * w; dR[1][2][2] = 2 * z; dR[1][2][3] = 2 * y;
    dR[2][0][0] = -2 * y; dR[2][0][1] = 2 * z; dR[2][0][2] = -2 * w; dR[2][0][3] = 2 * x;
    dR[2][1][0] = 2 * x;  dR[2][1][1] = 2 * w; dR[2][1][2] = 2 * z; dR[2][1][3] = 2 * y;
    dR[2][2][1] = -4 * x; dR[2][2][2] = -4 * y;
}

static void compute_geom(int i, const double* means, const double* log_scales, const double* quats,
                         const double* opacity_raw, const orc_cam* cam, geom* g)
{
    for (int k = 0; k < 3; ++k) g->p[k] = means[3 * i + k];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) g->Vr[r][c] = cam->view[4 * r + c];
    for (int r = 0; r < 3; ++r)
        g->t[r] = g->Vr[r][0] * g->p[0] + g->Vr[r][1] * g->p[1] + g->Vr[r][2] * g->p[2] + cam->view[4 * r + 3];
    for (int k = 0; k < 3; ++k) g->s[k] = exp(log_scales[3 * i + k]);
    double qr[4], n2 = 0;
    for (int k = 0; k < 4; ++k) {
        qr[k] = quats[4 * i + k];
        n2 += qr[k] * qr[k];
    }
    g->qnorm = sqrt(n2);
    for (int k = 0; k < 4; ++k) g->q[k] = qr[k] / g->qnorm;
    quat_rot(g->q, g->R);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) g->M[r][c] = g->R[r][c] * g->s[c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double v = 0;
            for (int k = 0; k < 3; ++k) v += g->M[r][k] * g->M[c][k];
            g->Sig[r][c] = v;
        }
    const double tz = g->t[2];
    g->xn = g->t[0] / tz;
    g->yn = g->t[1] / tz;
    const double limx = 1.3 * (0.5 * cam->W / (double)cam->fx);
    const double limy = 1.3 * (0.5 * cam->H / (double)cam->fy);
    g->clamped_x = !(g->xn >= -limx && g->xn <= limx);
    g->clamped_y = !(g->yn >= -limy && g->yn <= limy);
    g->xc = g->clamped_x ? (g->xn < 0 ? -limx : limx) : g->xn;
    g->yc = g->clamped_y ? (g->yn < 0 ? -limy : limy) : g->yn;
    memset(g->J, 0, sizeof g->J);
    g->J[0][0] = cam->fx / tz;
    g->J[0][2] = -cam->fx * g->xc / tz;
    g->J[1][1] = cam->fy / tz;
    g->J[1][2] = -cam->fy * g->yc / tz;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double v = 0;
            for (int k = 0; k < 3; ++k) v += g->J[r][k] * g->Vr[k][c];
            g->T[r][c] = v;
        }
    double S2[2][2];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double v = 0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) v += g->T[r][k] * g->Sig[k][l] * g->T[c][l];
            S2[r][c] = v;
        }
    g->a = S2[0][0] + 0.3;
    g->b = S2[0][1];
    g->c = S2[1][1] + 0.3;
    g->det = g->a * g->c - g->b * g->b;
    g->conic[0] = g->c / g->det;
    g->conic[1] = -g->b / g->det;
    g->conic[2] = g->a / g->det;
    g->o = 1.0 / (1.0 + exp(-opacity_raw[i]));
    double v[3], l2 = 0;
    for (int k = 0; k < 3; ++k) {
        v[k] = g->p[k] - cam->campos[k];
        l2 += v[k] * v[k];
    }
    g->vlen = sqrt(l2);
    for (int k = 0; k < 3; ++k) g->dir[k] = v[k] / g->vlen;
}

void orc_project(int N, int deg, const double* means, const double* log_scales, const double* quats,
                 const double* opacity_raw, const double* sh, const orc_cam* cam, const int32_t* tiles,
                 double* mean2d, double* depth, double* cov2d, double* conic, double* opacity,
                 double* rgb, uint8_t* clamp)
{
    const int nc = orc_sh_count(deg);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        mean2d[2 * i] = mean2d[2 * i + 1] = 0;
        depth[i] = 0;
        for (int k = 0; k < 3; ++k) cov2d[3 * i + k] = conic[3 * i + k] = rgb[3 * i + k] = 0;
        opacity[i] = 0;
        clamp[i] = 0;
        if (tiles[i] <= 0) continue;
        geom g;
        compute_geom(i, means, log_scales, quats, opacity_raw, cam, &g);
        mean2d[2 * i] = cam->fx * g.xn + cam->cx;
        mean2d[2 * i + 1] = cam->fy * g.yn + cam->cy;
        depth[i] = g.t[2];
        cov2d[3 * i] = g.a;
        cov2d[3 * i + 1] = g.b;
        cov2d[3 * i + 2] = g.c;
        for (int k = 0; k < 3; ++k) conic[3 * i + k] = g.conic[k];
        opacity[i] = g.o;
        double Y[16];
        orc_sh_basis(deg, g.dir, Y, NULL);
        uint8_t cm = 0;
        for (int ch = 0; ch < 3; ++ch) {
            double v = 0.5;
            for (int k = 0; k < nc; ++k) v += Y[k] * sh[((size_t)i * nc + k) * 3 + ch];
            if (v < 0) {
                cm |= (uint8_t)(1u << ch);
                v = 0;
            }
            rgb[3 * i + ch] = v;
        }
        clamp[i] = cm;
    }
}

void orc_project_bwd(int N, int deg, const double* means, const double* log_scales, const double* quats,
                     const double* opacity_raw, const double* sh, const orc_cam* cam, const int32_t* tiles,
                     const double* d_mean2d, const double* d_conic, const double* d_opacity,
                     const double* d_rgb, double* d_means, double* d_log_scales, double* d_quats,
                     double* d_opacity_raw, double* d_sh)
{
    const int nc = orc_sh_count(deg);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        for (int k = 0; k < 3; ++k) d_means[3 * i + k] = d_log_scales[3 * i + k] = 0;
        for (int k = 0; k < 4; ++k) d_quats[4 * i + k] = 0;
        d_opacity_raw[i] = 0;
        for (int k = 0; k < nc * 3; ++k) d_sh[(size_t)i * nc * 3 + k] = 0;
        if (tiles[i] <= 0) continue;
        geom g;
        compute_geom(i, means, log_scales, quats, opacity_raw, cam, &g);
        double Gp[3] = {0, 0, 0}, Gt[3] = {0, 0, 0};

        /* opacity */
        d_opacity_raw[i] = d_opacity[i] * g.o * (1 - g.o);

        /* colour: rgb_c = sum_k Y_k sh_kc + 0.5 unless clamped */
        double Y[16], dY[48];
        orc_sh_basis(deg, g.dir, Y, dY);
        double Gc[3], rgbv[3];
        for (int ch = 0; ch < 3; ++ch) {
            double v = 0.5;
            for (int k = 0; k < nc; ++k) v += Y[k] * sh[((size_t)i * nc + k) * 3 + ch];
            rgbv[ch] = v;
            Gc[ch] = (v < 0) ? 0.0 : d_rgb[3 * i + ch];
        }
        double Gdir[3] = {0, 0, 0};
        for (int k = 0; k < nc; ++k)
            for (int ch = 0; ch < 3; ++ch) {
                const double coef = sh[((size_t)i * nc + k) * 3 + ch];
                d_sh[((size_t)i * nc + k) * 3 + ch] = Y[k] * Gc[ch];
                for (int e = 0; e < 3; ++e) Gdir[e] += Gc[ch] * coef * dY[3 * k + e];
            }
        double dd = 0;
        for (int e = 0; e < 3; ++e) dd += g.dir[e] * Gdir[e];
        for (int e = 0; e < 3; ++e) Gp[e] += (Gdir[e] - g.dir[e] * dd) / g.vlen;

        /* conic (A, B, C) -> (a, b, c) */
        const double A = g.conic[0], B = g.conic[1], C = g.conic[2];
        const double dA = d_conic[3 * i], dB = d_conic[3 * i + 1], dC = d_conic[3 * i + 2];
        const double ga = -(dA * A * A + dB * A * B + dC * B * B);
        const double gb = -(2 * dA * A * B + dB * (A * C + B * B) + 2 * dC * B * C);
        const double gc = -(dA * B * B + dB * B * C + dC * C * C);

        /* (a, b, c) = (T0 S T0, T0 S T1, T1 S T1) -> dL/dSigma, dL/dT */
        double GS[3][3], GT[2][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                GS[r][c] = ga * g.T[0][r] * g.T[0][c] + gb * g.T[0][r] * g.T[1][c] + gc * g.T[1][r] * g.T[1][c];
        double ST0[3], ST1[3];
        for (int r = 0; r < 3; ++r) {
            ST0[r] = ST1[r] = 0;
            for (int k = 0; k < 3; ++k) {
                ST0[r] += g.Sig[r][k] * g.T[0][k];
                ST1[r] += g.Sig[r][k] * g.T[1][k];
            }
        }
        for (int r = 0; r < 3; ++r) {
            GT[0][r] = 2 * ga * ST0[r] + gb * ST1[r];
            GT[1][r] = gb * ST0[r] + 2 * gc * ST1[r];
        }
        /* T = J R_c -> dL/dJ */
        double GJ[2][3];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k) {
                double v = 0;
                for (int c = 0; c < 3; ++c) v += GT[r][c] * g.Vr[k][c];
                GJ[r][k] = v;
            }
        const double tz = g.t[2], fx = cam->fx, fy = cam->fy;
        /* J entries as functions of t (xc, yc held, then chained if not clamped) */
        Gt[2] += GJ[0][0] * (-fx / (tz * tz)) + GJ[1][1] * (-fy / (tz * tz)) +
                 GJ[0][2] * (fx * g.xc / (tz * tz)) + GJ[1][2] * (fy * g.yc / (tz * tz));
        const double Gxc = GJ[0][2] * (-fx / tz);
        const double Gyc = GJ[1][2] * (-fy / tz);
        if (!g.clamped_x) {
            Gt[0] += Gxc / tz;
            Gt[2] += -Gxc * g.t[0] / (tz * tz);
        }
        if (!g.clamped_y) {
            Gt[1] += Gyc / tz;
            Gt[2] += -Gyc * g.t[1] / (tz * tz);
        }
        /* mean2d */
        const double dmx = d_mean2d[2 * i], dmy = d_mean2d[2 * i + 1];
        Gt[0] += dmx * fx / tz;
        Gt[2] += -dmx * fx * g.t[0] / (tz * tz);
        Gt[1] += dmy * fy / tz;
        Gt[2] += -dmy * fy * g.t[1] / (tz * tz);
        /* t = R_c p + t_c */
        for (int k = 0; k < 3; ++k)
            for (int r = 0; r < 3; ++r) Gp[k] += g.Vr[r][k] * Gt[r];
        for (int k = 0; k < 3; ++k) d_means[3 * i + k] = Gp[k];

        /* Sigma = M M^T -> dL/dM = (GS + GS^T) M */
        double GM[3][3];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double v = 0;
                for (int k = 0; k < 3; ++k) v += (GS[r][k] + GS[k][r]) * g.M[k][c];
                GM[r][c] = v;
            }
        /* M = R diag(s) */
        double GR[3][3];
        for (int j = 0; j < 3; ++j) {
            double gs = 0;
            for (int r = 0; r < 3; ++r) {
                GR[r][j] = GM[r][j] * g.s[j];
                gs += GM[r][j] * g.R[r][j];
            }
            d_log_scales[3 * i + j] = gs * g.s[j];
        }
        /* R(q), q = q_raw / |q_raw| */
        double dR[3][3][4], Gq[4] = {0, 0, 0, 0};
        quat_rot_jac(g.q, dR);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                for (int k = 0; k < 4; ++k) Gq[k] += GR[r][c] * dR[r][c][k];
        double qg = 0;
        for (int k = 0; k < 4; ++k) qg += g.q[k] * Gq[k];
        for (int k = 0; k < 4; ++k) d_quats[4 * i + k] = (Gq[k] - g.q[k] * qg) / g.qnorm;
        (void)rgbv;
    }
}
