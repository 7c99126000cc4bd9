// Projection of 3D Gaussians to screen-space splats and its adjoint.
//
// Forward: Eq. 1 (eq:render) of the paper -- the attributes p, Sigma, c,
// alpha of every Gaussian are projected with the 3DGS EWA splatting model
// that Sec. 4 says the method reuses; s_G (Sec. 3.4.1) and u (Sec. 3.4.2) are
// copied into the 80-byte splat record the renderer reads.
// Backward: the exact adjoint (branch taken at the guard band and colour clamps).
//
// One thread per Gaussian.  Loads are coalesced across the warp; SH
// coefficients (192 B per Gaussian at degree 3) and the semantic feature are
// read with 16-byte vector loads, the splat record is written as 5 x float4.
#include "common.cuh"

namespace leg {
namespace {

// ----------------------------------------------------------------------------
// Key path: depth, screen mean, 2D covariance, radius and tile rectangle must
// be identical on every implementation, so they are computed with explicit
// round-to-nearest intrinsics (never contracted into FMAs by the compiler)
// in one fixed order.

// exp(x) in FP32 by Cody-Waite reduction (ln2 split into a 16-bit head and a
// tail) and the degree-7 Taylor polynomial of e^r on |r| <= ln2/2 in Horner
// form with fused multiply-adds, scaled by 2^n built from its bit pattern.
__device__ __forceinline__ float kp_exp(float x)
{
    x = fminf(fmaxf(x, -80.f), 80.f);
    const float n = rintf(__fmul_rn(x, 0x1.715476p+0f));
    float r = __fmaf_rn(-n, 0x1.62e4p-1f, x);
    r = __fmaf_rn(-n, 0x1.7f7d1cp-20f, r);
    float p = 0x1.a01a02p-13f;
    p = __fmaf_rn(p, r, 0x1.6c16c2p-10f);
    p = __fmaf_rn(p, r, 0x1.111112p-7f);
    p = __fmaf_rn(p, r, 0x1.555556p-5f);
    p = __fmaf_rn(p, r, 0x1.555556p-3f);
    p = __fmaf_rn(p, r, 0x1p-1f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    return __fmul_rn(p, __int_as_float(((int)n + 127) << 23));
}

__device__ __forceinline__ float dot3(float a0, float b0, float a1, float b1, float a2, float b2)
{
    return __fmaf_rn(a0, b0, __fmaf_rn(a1, b1, __fmul_rn(a2, b2)));
}

struct KeyGeom {
    float tx, ty, tz, xn, yn, xc, yc, inv_tz;
    float s[3], q[4], qnorm_inv, R[3][3], M[3][3], S[3][3], T0[3], T1[3];
    float a, b, c, det, mx, my, rf;
    float limx, limy;
    int radius, x0, y0, x1, y1;
    bool visible;
};

__device__ __forceinline__ void key_geometry(const CamParams& cam, float px, float py, float pz, const float* ls,
                                             const float* quat, KeyGeom& g)
{
    const float* V = cam.view;
    g.tx = __fmaf_rn(V[0], px, __fmaf_rn(V[1], py, __fmaf_rn(V[2], pz, V[3])));
    g.ty = __fmaf_rn(V[4], px, __fmaf_rn(V[5], py, __fmaf_rn(V[6], pz, V[7])));
    g.tz = __fmaf_rn(V[8], px, __fmaf_rn(V[9], py, __fmaf_rn(V[10], pz, V[11])));
    g.visible = false;
    g.radius = 0;
    g.x0 = g.y0 = g.x1 = g.y1 = 0;
    if (!(g.tz > cam.near_z)) return;

    for (int k = 0; k < 3; ++k) g.s[k] = kp_exp(ls[k]);
    float qw = quat[0], qx = quat[1], qy = quat[2], qz = quat[3];
    const float n2 = __fmaf_rn(qw, qw, __fmaf_rn(qx, qx, __fmaf_rn(qy, qy, __fmul_rn(qz, qz))));
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
    g.qnorm_inv = inv;
    qw = __fmul_rn(qw, inv);
    qx = __fmul_rn(qx, inv);
    qy = __fmul_rn(qy, inv);
    qz = __fmul_rn(qz, inv);
    g.q[0] = qw; g.q[1] = qx; g.q[2] = qy; g.q[3] = qz;
    const float xx = __fmul_rn(qx, qx), yy = __fmul_rn(qy, qy), zz = __fmul_rn(qz, qz);
    const float xy = __fmul_rn(qx, qy), xz = __fmul_rn(qx, qz), yz = __fmul_rn(qy, qz);
    const float wx = __fmul_rn(qw, qx), wy = __fmul_rn(qw, qy), wz = __fmul_rn(qw, qz);
    g.R[0][0] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(yy, zz)));
    g.R[0][1] = __fmul_rn(2.f, __fsub_rn(xy, wz));
    g.R[0][2] = __fmul_rn(2.f, __fadd_rn(xz, wy));
    g.R[1][0] = __fmul_rn(2.f, __fadd_rn(xy, wz));
    g.R[1][1] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(xx, zz)));
    g.R[1][2] = __fmul_rn(2.f, __fsub_rn(yz, wx));
    g.R[2][0] = __fmul_rn(2.f, __fsub_rn(xz, wy));
    g.R[2][1] = __fmul_rn(2.f, __fadd_rn(yz, wx));
    g.R[2][2] = __fsub_rn(1.f, __fmul_rn(2.f, __fadd_rn(xx, yy)));
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) g.M[r][c] = __fmul_rn(g.R[r][c], g.s[c]);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = r; c < 3; ++c) {
            g.S[r][c] = dot3(g.M[r][0], g.M[c][0], g.M[r][1], g.M[c][1], g.M[r][2], g.M[c][2]);
            g.S[c][r] = g.S[r][c];
        }

    g.inv_tz = __fdiv_rn(1.0f, g.tz);
    g.xn = __fmul_rn(g.tx, g.inv_tz);
    g.yn = __fmul_rn(g.ty, g.inv_tz);
    g.limx = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, (float)cam.W), cam.fx));
    g.limy = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, (float)cam.H), cam.fy));
    g.xc = fminf(fmaxf(g.xn, -g.limx), g.limx);
    g.yc = fminf(fmaxf(g.yn, -g.limy), g.limy);
    const float J00 = __fmul_rn(cam.fx, g.inv_tz);
    const float J02 = __fmul_rn(-__fmul_rn(cam.fx, g.xc), g.inv_tz);
    const float J11 = __fmul_rn(cam.fy, g.inv_tz);
    const float J12 = __fmul_rn(-__fmul_rn(cam.fy, g.yc), g.inv_tz);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        g.T0[j] = __fmaf_rn(J00, V[j], __fmul_rn(J02, V[8 + j]));
        g.T1[j] = __fmaf_rn(J11, V[4 + j], __fmul_rn(J12, V[8 + j]));
    }
    float U0[3], U1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        U0[k] = dot3(g.T0[0], g.S[0][k], g.T0[1], g.S[1][k], g.T0[2], g.S[2][k]);
        U1[k] = dot3(g.T1[0], g.S[0][k], g.T1[1], g.S[1][k], g.T1[2], g.S[2][k]);
    }
    g.a = __fadd_rn(dot3(U0[0], g.T0[0], U0[1], g.T0[1], U0[2], g.T0[2]), 0.3f);
    g.b = dot3(U0[0], g.T1[0], U0[1], g.T1[1], U0[2], g.T1[2]);
    g.c = __fadd_rn(dot3(U1[0], g.T1[0], U1[1], g.T1[1], U1[2], g.T1[2]), 0.3f);
    g.det = __fmaf_rn(g.a, g.c, -__fmul_rn(g.b, g.b));
    if (!(g.det > 0.f)) return;

    g.mx = __fmaf_rn(cam.fx, g.xn, cam.cx);
    g.my = __fmaf_rn(cam.fy, g.yn, cam.cy);
    const float mid = __fmul_rn(0.5f, __fadd_rn(g.a, g.c));
    const float disc = fmaxf(0.1f, __fmaf_rn(mid, mid, -g.det));
    const float lam = __fadd_rn(mid, __fsqrt_rn(disc));
    const float rf = fminf(ceilf(__fmul_rn(3.0f, __fsqrt_rn(lam))), 1048576.0f);
    const float TXf = (float)cam.TX, TYf = (float)cam.TY;
    g.x0 = (int)fminf(fmaxf(floorf(__fmul_rn(__fsub_rn(g.mx, rf), 0.0625f)), 0.f), TXf);
    g.x1 = (int)fminf(fmaxf(floorf(__fmul_rn(__fadd_rn(__fadd_rn(g.mx, rf), 15.0f), 0.0625f)), 0.f), TXf);
    g.y0 = (int)fminf(fmaxf(floorf(__fmul_rn(__fsub_rn(g.my, rf), 0.0625f)), 0.f), TYf);
    g.y1 = (int)fminf(fmaxf(floorf(__fmul_rn(__fadd_rn(__fadd_rn(g.my, rf), 15.0f), 0.0625f)), 0.f), TYf);
    if ((g.x1 - g.x0) * (g.y1 - g.y0) <= 0) return;
    g.radius = (int)rf;
    g.rf = rf;
    g.visible = true;
}

// Upper bound of ln(x), normal x > 0, within 0.0141 of it: x = m 2^e with m in
// [1, 2) taken from the bit pattern, and ln m <= (m - 1)/sqrt(m) for m >= 1
// (equality at m = 1; the gap grows to 1/sqrt(2) - ln 2 at m = 2).
__device__ __forceinline__ float kp_ln_up(float x)
{
    const uint32_t bits = __float_as_uint(x);
    const int e = (int)(bits >> 23) - 127;
    const float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);
    return __fadd_rn(__fmul_rn((float)e, 0x1.62e430p-1f), __fdiv_rn(__fsub_rn(m, 1.0f), __fsqrt_rn(m)));
}

// Tile ellipse of a visible Gaussian (key path; binning uses it to skip the
// rect tiles it cannot reach).  Pixels with o exp(-q/2) >= 1/255 satisfy
// q <= 2 ln(255 o); t bounds that from above with a margin of 1/16 and a factor
// 1 + 2^-10 that absorb the rounding of o, the conic and the renderer's exp.
// Stored as {mx, my, s, k} {mm, ystar, padx, pady}: a row at offset dy spans
// dx in s dy -+ sqrt(k (mm - dy^2)), mm = c t is the squared half-height and
// ystar = b sqrt(t/a) the row offset of the right-most point; the pads (in
// pixels) cover the rounding of the span arithmetic.
__device__ __forceinline__ void key_ellipse(const KeyGeom& g, float opacity_raw, float4& e0, float4& e1)
{
    const float o = __fdiv_rn(1.0f, __fadd_rn(1.0f, kp_exp(-opacity_raw)));
    const float t = __fmul_rn(__fadd_rn(__fmul_rn(2.0f, kp_ln_up(__fmul_rn(255.0f, o))), 0.0625f), 1.0009765625f);
    e0 = make_float4(g.mx, g.my, 0.f, 0.f);
    e1 = make_float4(-1.0f, 0.f, 0.f, 0.f);
    if (t > 0.f) {
        e0.z = __fdiv_rn(g.b, g.c);
        e0.w = __fdiv_rn(g.det, __fmul_rn(g.c, g.c));
        e1.x = __fmul_rn(g.c, t);
        e1.y = __fmul_rn(g.b, __fsqrt_rn(__fdiv_rn(t, g.a)));
    }
    const float r2 = __fmul_rn(2.0f, g.rf);
    e1.z = __fadd_rn(0.25f, __fmul_rn(__fadd_rn(fabsf(g.mx), r2), 0x1p-12f));
    e1.w = __fadd_rn(0.25f, __fmul_rn(__fadd_rn(fabsf(g.my), r2), 0x1p-12f));
}

// ----------------------------------------------------------------------------
// Real spherical harmonics up to degree 3, coefficient k = l^2 + l + m, with
// the Condon-Shortley phase, as polynomials in the unit direction (x, y, z);
// dY = their Cartesian gradient (projected onto the sphere by the caller).
constexpr float SH_C0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float SH_C1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float SH_C2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float SH_C2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float SH_C2c = 0.5462742152960396f;   // sqrt(15/pi)/4
constexpr float SH_C3a = 0.5900435899266435f;   // sqrt(35/(2 pi))/4
constexpr float SH_C3b = 2.890611442640554f;    // sqrt(105/pi)/2
constexpr float SH_C3c = 0.4570457994644658f;   // sqrt(21/(2 pi))/4
constexpr float SH_C3d = 0.3731763325901154f;   // sqrt(7/pi)/4
constexpr float SH_C3e = 1.445305721320277f;    // sqrt(105/pi)/4

template <bool GRAD>
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y, float (*dY)[3])
{
    Y[0] = SH_C0;
    if (GRAD) dY[0][0] = dY[0][1] = dY[0][2] = 0.f;
    if (deg < 1) return;
    Y[1] = -SH_C1 * y;
    Y[2] = SH_C1 * z;
    Y[3] = -SH_C1 * x;
    if (GRAD) {
        dY[1][0] = 0.f; dY[1][1] = -SH_C1; dY[1][2] = 0.f;
        dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = SH_C1;
        dY[3][0] = -SH_C1; dY[3][1] = 0.f; dY[3][2] = 0.f;
    }
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = SH_C2a * x * y;
    Y[5] = -SH_C2a * y * z;
    Y[6] = SH_C2b * (3.f * zz - 1.f);
    Y[7] = -SH_C2a * x * z;
    Y[8] = SH_C2c * (xx - yy);
    if (GRAD) {
        dY[4][0] = SH_C2a * y; dY[4][1] = SH_C2a * x; dY[4][2] = 0.f;
        dY[5][0] = 0.f; dY[5][1] = -SH_C2a * z; dY[5][2] = -SH_C2a * y;
        dY[6][0] = 0.f; dY[6][1] = 0.f; dY[6][2] = 6.f * SH_C2b * z;
        dY[7][0] = -SH_C2a * z; dY[7][1] = 0.f; dY[7][2] = -SH_C2a * x;
        dY[8][0] = 2.f * SH_C2c * x; dY[8][1] = -2.f * SH_C2c * y; dY[8][2] = 0.f;
    }
    if (deg < 3) return;
    Y[9] = -SH_C3a * (3.f * xx - yy) * y;
    Y[10] = SH_C3b * x * y * z;
    Y[11] = -SH_C3c * y * (5.f * zz - 1.f);
    Y[12] = SH_C3d * z * (5.f * zz - 3.f);
    Y[13] = -SH_C3c * x * (5.f * zz - 1.f);
    Y[14] = SH_C3e * (xx - yy) * z;
    Y[15] = -SH_C3a * (xx - 3.f * yy) * x;
    if (GRAD) {
        dY[9][0] = -6.f * SH_C3a * x * y; dY[9][1] = -3.f * SH_C3a * (xx - yy); dY[9][2] = 0.f;
        dY[10][0] = SH_C3b * y * z; dY[10][1] = SH_C3b * x * z; dY[10][2] = SH_C3b * x * y;
        dY[11][0] = 0.f; dY[11][1] = -SH_C3c * (5.f * zz - 1.f); dY[11][2] = -10.f * SH_C3c * y * z;
        dY[12][0] = 0.f; dY[12][1] = 0.f; dY[12][2] = SH_C3d * (15.f * zz - 3.f);
        dY[13][0] = -SH_C3c * (5.f * zz - 1.f); dY[13][1] = 0.f; dY[13][2] = -10.f * SH_C3c * x * z;
        dY[14][0] = 2.f * SH_C3e * x * z; dY[14][1] = -2.f * SH_C3e * y * z; dY[14][2] = SH_C3e * (xx - yy);
        dY[15][0] = -3.f * SH_C3a * (xx - yy); dY[15][1] = 6.f * SH_C3a * x * y; dY[15][2] = 0.f;
    }
}

// SH coefficients of Gaussian i into registers ([k][3]); 16-byte vector loads
// when the per-Gaussian stride allows it (degrees 1 and 3).
// RO: through the read-only data path (only where nothing writes sh during the kernel).
template <bool RO = true>
__device__ __forceinline__ void load_sh(const float* sh, int i, int nc, float* out)
{
    const size_t base = (size_t)i * nc * 3;
    if ((nc * 3) % 4 == 0) {
        const float4* p = reinterpret_cast<const float4*>(sh + base);
        for (int v = 0; v < nc * 3 / 4; ++v) {
            const float4 t = RO ? __ldg(p + v) : p[v];
            out[4 * v] = t.x;
            out[4 * v + 1] = t.y;
            out[4 * v + 2] = t.z;
            out[4 * v + 3] = t.w;
        }
    } else {
        for (int k = 0; k < nc * 3; ++k) out[k] = RO ? __ldg(sh + base + k) : sh[base + k];
    }
}

template <int DEG>
__global__ void __launch_bounds__(256) preprocess_kernel(int n, const float* __restrict__ means,
                                                         const float* __restrict__ log_scales,
                                                         const float* __restrict__ quats,
                                                         const float* __restrict__ opacity_raw,
                                                         const float* __restrict__ sh,
                                                         const float* __restrict__ feat,
                                                         const float* __restrict__ unc, CamParams cam,
                                                         float4* __restrict__ splat, float* __restrict__ depth,
                                                         int* __restrict__ radius, ushort4* __restrict__ rect,
                                                         int* __restrict__ tiles, uint8_t* __restrict__ clamp,
                                                         float4* __restrict__ ellipse)
{
    constexpr int NC = (DEG + 1) * (DEG + 1);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float px = __ldg(means + 3 * i), py = __ldg(means + 3 * i + 1), pz = __ldg(means + 3 * i + 2);
    float ls[3], q[4];
    for (int k = 0; k < 3; ++k) ls[k] = __ldg(log_scales + 3 * i + k);
    const float4 q4 = __ldg(reinterpret_cast<const float4*>(quats) + i);
    q[0] = q4.x; q[1] = q4.y; q[2] = q4.z; q[3] = q4.w;
    KeyGeom g;
    key_geometry(cam, px, py, pz, ls, q, g);
    depth[i] = g.tz;
    float4* rec = splat + (size_t)i * 5;
    if (!g.visible) {
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = 0; k < 5; ++k) rec[k] = z4;
        radius[i] = 0;
        rect[i] = make_ushort4(0, 0, 0, 0);
        tiles[i] = 0;
        clamp[i] = 0;
        ellipse[2 * i] = z4;
        ellipse[2 * i + 1] = z4;
        return;
    }
    {
        float4 e0, e1;
        key_ellipse(g, __ldg(opacity_raw + i), e0, e1);
        ellipse[2 * i] = e0;
        ellipse[2 * i + 1] = e1;
    }
    const float inv_det = 1.0f / g.det;
    const float A = g.c * inv_det, B = -g.b * inv_det, C = g.a * inv_det;
    const float op = 1.0f / (1.0f + expf(-__ldg(opacity_raw + i)));

    float dx = px - cam.campos[0], dy = py - cam.campos[1], dz = pz - cam.campos[2];
    const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= il; dy *= il; dz *= il;
    float Y[16];
    sh_basis<false>(DEG, dx, dy, dz, Y, nullptr);
    float coef[NC * 3];
    load_sh(sh, i, NC, coef);
    float col[3];
    uint8_t cm = 0;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float v = 0.5f;
#pragma unroll
        for (int k = 0; k < NC; ++k) v = fmaf(Y[k], coef[3 * k + ch], v);
        if (v < 0.f) {
            cm |= (uint8_t)(1u << ch);
            v = 0.f;
        }
        col[ch] = v;
    }
    const float4 f0 = __ldg(reinterpret_cast<const float4*>(feat) + 2 * i);
    const float4 f1 = __ldg(reinterpret_cast<const float4*>(feat) + 2 * i + 1);
    rec[0] = make_float4(g.mx, g.my, A * kConicScaleAC, B * kConicScaleB);
    rec[1] = make_float4(C * kConicScaleAC, op, col[0], col[1]);
    rec[2] = make_float4(col[2], __ldg(unc + i), f0.x, f0.y);
    rec[3] = make_float4(f0.z, f0.w, f1.x, f1.y);
    rec[4] = make_float4(f1.z, f1.w, 0.f, 0.f);
    radius[i] = g.radius;
    rect[i] = make_ushort4((unsigned short)g.x0, (unsigned short)g.y0, (unsigned short)g.x1, (unsigned short)g.y1);
    tiles[i] = (g.x1 - g.x0) * (g.y1 - g.y0);
    clamp[i] = cm;
}

// ----------------------------------------------------------------------------
// Backward of the projection.  Each thread computes the parameter gradients of
// one Gaussian into a per-warp staging area in shared memory (Gaussian-major,
// in each field's own layout; the SH gradient Y_k dL/drgb_c is kept factored
// as the basis Y and the colour gradient).  Each warp then hands the
// contiguous ranges of its 32 Gaussians to the sink with coalesced 16-byte
// accesses: GradSink stores the gradients, AdamSink applies one Adam step to
// parameters and moments in place, so the gradients never reach memory.
template <int NC>
struct GradStage {
    float means[32 * 3], scales[32 * 3], quats[32 * 4], opacity[32], feat[32 * 8], unc[32];
    float Y[32 * NC], gcol[32 * 3];
};

enum { kFMeans, kFScales, kFQuats, kFOpacity, kFSH, kFFeat, kFUnc };

// Gradient of element e of the warp's sh range.
template <int NC>
__device__ __forceinline__ float sh_grad(const GradStage<NC>& S, int e)
{
    const int gi = e / (NC * 3), r = e - gi * (NC * 3), k = r / 3;
    return S.Y[gi * NC + k] * S.gcol[gi * 3 + (r - 3 * k)];
}

// Elements [0, len) of the warp's range of one field, starting at flat index
// base of that field; grad(e) gives element e's gradient.  16-byte accesses
// where the sink's arrays are 16-byte aligned at base (base is a multiple of
// 4), two of them in flight per lane; the n % 4 tail element by element.
template <class Sink, class GradOf>
__device__ __forceinline__ void warp_apply(const Sink& sk, int f, size_t base, int len, int lane, float lo, float hi,
                                           const GradOf& grad)
{
    int e0 = 0;
    if (sk.aligned(f, base)) {
        const int len4 = len & ~3;
        for (int e = 4 * lane; e < len4; e += 256) {
            const float4 ga = make_float4(grad(e), grad(e + 1), grad(e + 2), grad(e + 3));
            if (e + 128 < len4) {
                const int e2 = e + 128;
                const float4 gb = make_float4(grad(e2), grad(e2 + 1), grad(e2 + 2), grad(e2 + 3));
                sk.put4x2(f, (base + e) >> 2, 32, ga, gb, lo, hi);
            } else {
                sk.put4(f, (base + e) >> 2, ga, lo, hi);
            }
        }
        e0 = len4;
    }
    for (int e = e0 + lane; e < len; e += 32) sk.put1(f, base + e, grad(e), lo, hi);
}

struct GradSink {
    static constexpr bool kExtra = false;
    float* d[7];
    __device__ __forceinline__ bool aligned(int f, size_t base) const
    {
        return ((reinterpret_cast<uintptr_t>(d[f] + base)) & 15u) == 0;
    }
    __device__ __forceinline__ void put1(int f, size_t i, float g, float, float) const { d[f][i] = g; }
    __device__ __forceinline__ void put4(int f, size_t i4, float4 g, float, float) const
    {
        reinterpret_cast<float4*>(d[f])[i4] = g;
    }
    __device__ __forceinline__ void put4x2(int f, size_t i4, int step4, float4 ga, float4 gb, float, float) const
    {
        reinterpret_cast<float4*>(d[f])[i4] = ga;
        reinterpret_cast<float4*>(d[f])[i4 + step4] = gb;
    }
};

struct AdamSink {
    static constexpr bool kExtra = true;
    float *p[7], *m[7], *v[7];
    AdamParams h;
    // one more flat range updated by the same step (no clamp), by the blocks
    // past the Gaussians' (gblocks): xp, xg, xm, xv of xn elements, 16-byte aligned
    float *xp = nullptr, *xm = nullptr, *xv = nullptr;
    const float* xg = nullptr;
    int64_t xn = 0;
    int gblocks = 0;
    // extra block b of nb: quads b * 128 + t, strided by nb * 128, then the xn % 4 tail
    __device__ __forceinline__ void extra(int b, int nb) const
    {
        const int64_t n4 = xn / 4, t = (int64_t)b * blockDim.x + threadIdx.x, stride = (int64_t)nb * blockDim.x;
        for (int64_t q = t; q < n4; q += stride) {
            float4 pp = reinterpret_cast<float4*>(xp)[q], mm = reinterpret_cast<float4*>(xm)[q];
            float4 vv = reinterpret_cast<float4*>(xv)[q];
            adam_step4(pp, reinterpret_cast<const float4*>(xg)[q], mm, vv, h, -INFINITY, INFINITY);
            reinterpret_cast<float4*>(xp)[q] = pp;
            reinterpret_cast<float4*>(xm)[q] = mm;
            reinterpret_cast<float4*>(xv)[q] = vv;
        }
        for (int64_t i = 4 * n4 + t; i < xn; i += stride) xp[i] = adam_step(xp[i], xg[i], xm[i], xv[i], h, -INFINITY, INFINITY);
    }
    __device__ __forceinline__ bool aligned(int f, size_t base) const
    {
        return ((reinterpret_cast<uintptr_t>(p[f] + base) | reinterpret_cast<uintptr_t>(m[f] + base) |
                 reinterpret_cast<uintptr_t>(v[f] + base)) & 15u) == 0;
    }
    __device__ __forceinline__ void put1(int f, size_t i, float g, float lo, float hi) const
    {
        float mm = m[f][i], vv = v[f][i];
        p[f][i] = adam_step(p[f][i], g, mm, vv, h, lo, hi);
        m[f][i] = mm;
        v[f][i] = vv;
    }
    __device__ __forceinline__ void put4(int f, size_t i4, float4 g, float lo, float hi) const
    {
        float4 pp = reinterpret_cast<float4*>(p[f])[i4], mm = reinterpret_cast<float4*>(m[f])[i4];
        float4 vv = reinterpret_cast<float4*>(v[f])[i4];
        adam_step4(pp, g, mm, vv, h, lo, hi);
        reinterpret_cast<float4*>(p[f])[i4] = pp;
        reinterpret_cast<float4*>(m[f])[i4] = mm;
        reinterpret_cast<float4*>(v[f])[i4] = vv;
    }
    // quads i4 and i4 + step4: all six loads issued before any store (the
    // three arrays are distinct, and nothing else touches them here)
    __device__ __forceinline__ void put4x2(int f, size_t i4, int step4, float4 ga, float4 gb, float lo,
                                           float hi) const
    {
        float4* __restrict__ P = reinterpret_cast<float4*>(p[f]);
        float4* __restrict__ M = reinterpret_cast<float4*>(m[f]);
        float4* __restrict__ V = reinterpret_cast<float4*>(v[f]);
        float4 pa = P[i4], ma = M[i4], va = V[i4];
        float4 pb = P[i4 + step4], mb = M[i4 + step4], vb = V[i4 + step4];
        adam_step4(pa, ga, ma, va, h, lo, hi);
        adam_step4(pb, gb, mb, vb, h, lo, hi);
        P[i4] = pa;
        M[i4] = ma;
        V[i4] = va;
        P[i4 + step4] = pb;
        M[i4 + step4] = mb;
        V[i4 + step4] = vb;
    }
};

// Adjoint of preprocess_kernel for Gaussian i, written into stage slot `lane`.
// Reads the screen-space gradient record (same layout as the splat record).
template <int DEG>
__device__ __forceinline__ void gaussian_grads(int i, int lane, const float* means, const float* log_scales,
                                               const float* quats, const float* opacity_raw, const float* sh,
                                               const CamParams& cam, const int* __restrict__ tiles,
                                               const uint8_t* __restrict__ clamp, const float4* __restrict__ grad2d,
                                               GradStage<(DEG + 1) * (DEG + 1)>& S)
{
    constexpr int NC = (DEG + 1) * (DEG + 1);
    const float4 g0 = grad2d[5 * (size_t)i], g1 = grad2d[5 * (size_t)i + 1], g2 = grad2d[5 * (size_t)i + 2];
    const float4 g3 = grad2d[5 * (size_t)i + 3], g4 = grad2d[5 * (size_t)i + 4];
    // semantic feature and uncertainty pass straight through
    reinterpret_cast<float4*>(S.feat)[2 * lane] = make_float4(g2.z, g2.w, g3.x, g3.y);
    reinterpret_cast<float4*>(S.feat)[2 * lane + 1] = make_float4(g3.z, g3.w, g4.x, g4.y);
    S.unc[lane] = g2.y;
    if (tiles[i] <= 0) {
        for (int k = 0; k < 3; ++k) S.means[3 * lane + k] = S.scales[3 * lane + k] = S.gcol[3 * lane + k] = 0.f;
        for (int k = 0; k < NC; ++k) S.Y[NC * lane + k] = 0.f;
        reinterpret_cast<float4*>(S.quats)[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        S.opacity[lane] = 0.f;
        return;
    }
    const float gmx = g0.x, gmy = g0.y, gA = g0.z, gB = g0.w, gC = g1.x, gop = g1.y;
    float gcol[3] = {g1.z, g1.w, g2.x};

    const float px = means[3 * i], py = means[3 * i + 1], pz = means[3 * i + 2];
    float ls[3], q[4];
    for (int k = 0; k < 3; ++k) ls[k] = log_scales[3 * i + k];
    const float4 q4 = reinterpret_cast<const float4*>(quats)[i];
    q[0] = q4.x; q[1] = q4.y; q[2] = q4.z; q[3] = q4.w;
    KeyGeom g;
    key_geometry(cam, px, py, pz, ls, q, g);

    // opacity
    const float op = 1.0f / (1.0f + expf(-opacity_raw[i]));
    S.opacity[lane] = gop * op * (1.f - op);

    // colour through SH and the view direction
    const uint8_t cm = clamp[i];
    for (int ch = 0; ch < 3; ++ch)
        if (cm & (1u << ch)) gcol[ch] = 0.f;
    float vx = px - cam.campos[0], vy = py - cam.campos[1], vz = pz - cam.campos[2];
    const float il = rsqrtf(vx * vx + vy * vy + vz * vz);
    const float dx = vx * il, dy = vy * il, dz = vz * il;
    float Y[16], dY[16][3];
    sh_basis<true>(DEG, dx, dy, dz, Y, dY);
    float coef[NC * 3];
    load_sh<false>(sh, i, NC, coef);
    float gdir[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        float w = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) w = fmaf(gcol[ch], coef[3 * k + ch], w);
        gdir[0] = fmaf(w, dY[k][0], gdir[0]);
        gdir[1] = fmaf(w, dY[k][1], gdir[1]);
        gdir[2] = fmaf(w, dY[k][2], gdir[2]);
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) S.Y[NC * lane + k] = Y[k];
    for (int ch = 0; ch < 3; ++ch) S.gcol[3 * lane + ch] = gcol[ch];
    const float dd = dx * gdir[0] + dy * gdir[1] + dz * gdir[2];
    float Gp[3] = {(gdir[0] - dx * dd) * il, (gdir[1] - dy * dd) * il, (gdir[2] - dz * dd) * il};

    // conic (A,B,C) = inverse of [[a,b],[b,c]]
    const float inv_det = 1.0f / g.det;
    const float A = g.c * inv_det, B = -g.b * inv_det, C = g.a * inv_det;
    const float ga = -(gA * A * A + gB * A * B + gC * B * B);
    const float gb = -(2.f * gA * A * B + gB * (A * C + B * B) + 2.f * gC * B * C);
    const float gc = -(gA * B * B + gB * B * C + gC * C * C);

    // (a, b, c) = (T0 S T0, T0 S T1, T1 S T1)
    float ST0[3], ST1[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        ST0[r] = g.S[r][0] * g.T0[0] + g.S[r][1] * g.T0[1] + g.S[r][2] * g.T0[2];
        ST1[r] = g.S[r][0] * g.T1[0] + g.S[r][1] * g.T1[1] + g.S[r][2] * g.T1[2];
    }
    float GT0[3], GT1[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        GT0[r] = 2.f * ga * ST0[r] + gb * ST1[r];
        GT1[r] = gb * ST0[r] + 2.f * gc * ST1[r];
    }
    // T = J R_c: only J00, J02, J11, J12 depend on t
    const float* V = cam.view;
    const float GJ00 = GT0[0] * V[0] + GT0[1] * V[1] + GT0[2] * V[2];
    const float GJ02 = GT0[0] * V[8] + GT0[1] * V[9] + GT0[2] * V[10];
    const float GJ11 = GT1[0] * V[4] + GT1[1] * V[5] + GT1[2] * V[6];
    const float GJ12 = GT1[0] * V[8] + GT1[1] * V[9] + GT1[2] * V[10];
    const float tz = g.tz, itz = 1.0f / tz, itz2 = itz * itz;
    const float fx = cam.fx, fy = cam.fy;
    float Gtx = 0.f, Gty = 0.f;
    float Gtz = GJ00 * (-fx * itz2) + GJ11 * (-fy * itz2) + GJ02 * (fx * g.xc * itz2) + GJ12 * (fy * g.yc * itz2);
    const float Gxc = GJ02 * (-fx * itz), Gyc = GJ12 * (-fy * itz);
    if (g.xn >= -g.limx && g.xn <= g.limx) {
        Gtx += Gxc * itz;
        Gtz -= Gxc * g.tx * itz2;
    }
    if (g.yn >= -g.limy && g.yn <= g.limy) {
        Gty += Gyc * itz;
        Gtz -= Gyc * g.ty * itz2;
    }
    // screen mean
    Gtx += gmx * fx * itz;
    Gty += gmy * fy * itz;
    Gtz -= (gmx * fx * g.tx + gmy * fy * g.ty) * itz2;
    // t = R_c p + t_c
#pragma unroll
    for (int k = 0; k < 3; ++k) Gp[k] += V[k] * Gtx + V[4 + k] * Gty + V[8 + k] * Gtz;
    for (int k = 0; k < 3; ++k) S.means[3 * lane + k] = Gp[k];

    // Sigma = M M^T: dL/dM = (GS + GS^T) M with GS = ga T0T0' + gb T0T1' + gc T1T1'
    float Gsym[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            Gsym[r][c] = 2.f * ga * g.T0[r] * g.T0[c] + gb * (g.T0[r] * g.T1[c] + g.T1[r] * g.T0[c]) +
                         2.f * gc * g.T1[r] * g.T1[c];
    float GR[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        float gs = 0.f;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float gm = Gsym[r][0] * g.M[0][j] + Gsym[r][1] * g.M[1][j] + Gsym[r][2] * g.M[2][j];
            GR[r][j] = gm * g.s[j];
            gs += gm * g.R[r][j];
        }
        S.scales[3 * lane + j] = gs * g.s[j];
    }
    // R(q), q = (w, x, y, z) normalised
    const float w = g.q[0], x = g.q[1], y = g.q[2], z = g.q[3];
    float Gq[4];
    Gq[0] = 2.f * (-z * GR[0][1] + y * GR[0][2] + z * GR[1][0] - x * GR[1][2] - y * GR[2][0] + x * GR[2][1]);
    Gq[1] = 2.f * (y * GR[0][1] + z * GR[0][2] + y * GR[1][0] - w * GR[1][2] + z * GR[2][0] + w * GR[2][1]) -
            4.f * x * (GR[1][1] + GR[2][2]);
    Gq[2] = 2.f * (x * GR[0][1] + w * GR[0][2] + x * GR[1][0] + z * GR[1][2] - w * GR[2][0] + z * GR[2][1]) -
            4.f * y * (GR[0][0] + GR[2][2]);
    Gq[3] = 2.f * (-w * GR[0][1] + x * GR[0][2] + w * GR[1][0] + y * GR[1][2] + x * GR[2][0] + y * GR[2][1]) -
            4.f * z * (GR[0][0] + GR[1][1]);
    const float qg = w * Gq[0] + x * Gq[1] + y * Gq[2] + z * Gq[3];
    const float qi = g.qnorm_inv;
    reinterpret_cast<float4*>(S.quats)[lane] =
        make_float4((Gq[0] - w * qg) * qi, (Gq[1] - x * qg) * qi, (Gq[2] - y * qg) * qi, (Gq[3] - z * qg) * qi);
}

// One thread per Gaussian, then one warp per 32 Gaussians for the sink.  The
// parameter pointers are not __restrict__: with AdamSink the kernel updates
// them (after the warp has read every value it needs: __syncwarp below).
// Eight blocks per SM (64 registers): the sink's loads wait on DRAM, and more
// resident warps hide that better than the few spills cost (1M Gaussians,
// SH degree 3, with Adam: 0.437 ms at 96 registers, 0.386 ms at 64).
template <int DEG, class Sink>
__global__ void __launch_bounds__(128, 8) preprocess_bwd_kernel(
    int n, const float* means, const float* log_scales, const float* quats, const float* opacity_raw, const float* sh,
    CamParams cam, const int* __restrict__ tiles, const uint8_t* __restrict__ clamp,
    const float4* __restrict__ grad2d, Sink sk)
{
    constexpr int NC = (DEG + 1) * (DEG + 1);
    constexpr float kInf = INFINITY;
    __shared__ GradStage<NC> stage[4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    GradStage<NC>& S = stage[w];
    if constexpr (Sink::kExtra) {
        if ((int)blockIdx.x >= sk.gblocks) {
            sk.extra((int)blockIdx.x - sk.gblocks, (int)gridDim.x - sk.gblocks);
            return;
        }
    }
    const int gw = blockIdx.x * 128 + 32 * w;
    if (gw >= n) return;
    const int i = gw + lane;
    if (i < n) gaussian_grads<DEG>(i, lane, means, log_scales, quats, opacity_raw, sh, cam, tiles, clamp, grad2d, S);
    __syncwarp();
    const int cnt = min(32, n - gw);
    const size_t g = (size_t)gw;
    warp_apply(sk, kFMeans, 3 * g, 3 * cnt, lane, -kInf, kInf, [&](int e) { return S.means[e]; });
    warp_apply(sk, kFScales, 3 * g, 3 * cnt, lane, -kInf, kInf, [&](int e) { return S.scales[e]; });
    warp_apply(sk, kFQuats, 4 * g, 4 * cnt, lane, -kInf, kInf, [&](int e) { return S.quats[e]; });
    warp_apply(sk, kFOpacity, g, cnt, lane, -kInf, kInf, [&](int e) { return S.opacity[e]; });
    warp_apply(sk, kFSH, (size_t)NC * 3 * g, NC * 3 * cnt, lane, -kInf, kInf,
               [&](int e) { return sh_grad<NC>(S, e); });
    warp_apply(sk, kFFeat, 8 * g, 8 * cnt, lane, -kInf, kInf, [&](int e) { return S.feat[e]; });
    warp_apply(sk, kFUnc, g, cnt, lane, 0.f, 1.f, [&](int e) { return S.unc[e]; });
}

}  // namespace

le_status check_gaussians(const le_gaussians* g)
{
    LE_CHECK_ARG(g != nullptr, "gaussians is null");
    LE_CHECK_ARG(g->n >= 0, "n = %d < 0", g->n);
    LE_CHECK_ARG(g->sh_degree >= 0 && g->sh_degree <= 3, "sh_degree %d not in 0..3", g->sh_degree);
    if (g->n == 0) return LE_OK;
    LE_CHECK_ARG(g->means && g->log_scales && g->quats && g->opacity_raw && g->sh && g->feat && g->unc,
                 "null Gaussian parameter pointer");
    LE_CHECK_ARG(aligned16(g->quats) && aligned16(g->sh) && aligned16(g->feat),
                 "quats, sh and feat must be 16-byte aligned");
    return LE_OK;
}

}  // namespace leg

using namespace leg;

extern "C" le_status le_preprocess(const le_gaussians* g, const le_camera* cam, le_projected* out, void* stream)
{
    LE_TRACE("le_preprocess");
    le_status st = check_gaussians(g);
    if (st != LE_OK) return st;
    if ((st = check_camera(cam)) != LE_OK) return st;
    LE_CHECK_ARG(out != nullptr, "projected is null");
    if (g->n == 0) return LE_OK;
    LE_CHECK_ARG(out->splat && out->depth && out->radius && out->rect && out->tiles_touched && out->clamp_mask &&
                     out->tile_ellipse,
                 "null projected pointer");
    LE_CHECK_ARG(aligned16(out->splat) && aligned16(out->tile_ellipse),
                 "splat and tile_ellipse must be 16-byte aligned");
    LE_CHECK_ARG(aligned16(out->rect) || (reinterpret_cast<uintptr_t>(out->rect) & 7u) == 0,
                 "rect must be 8-byte aligned");
    const CamParams cp = cam_params(cam);
    const int threads = 256, blocks = (g->n + threads - 1) / threads;
    cudaStream_t s = as_stream(stream);
#define LE_PRE(DEG)                                                                                         \
    preprocess_kernel<DEG><<<blocks, threads, 0, s>>>(g->n, g->means, g->log_scales, g->quats, g->opacity_raw, \
                                                      g->sh, g->feat, g->unc, cp,                            \
                                                      reinterpret_cast<float4*>(out->splat), out->depth,     \
                                                      out->radius, reinterpret_cast<ushort4*>(out->rect),    \
                                                      out->tiles_touched, out->clamp_mask,                   \
                                                      reinterpret_cast<float4*>(out->tile_ellipse))
    switch (g->sh_degree) {
        case 0: LE_PRE(0); break;
        case 1: LE_PRE(1); break;
        case 2: LE_PRE(2); break;
        default: LE_PRE(3); break;
    }
#undef LE_PRE
    LE_LAUNCHED();
    return LE_OK;
}

namespace leg {
template <class Sink>
static le_status launch_preprocess_backward(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                                            const float* grad2d, const Sink& sk, cudaStream_t s)
{
    const CamParams cp = cam_params(cam);
    const int threads = 128, gblocks = (g->n + threads - 1) / threads;
    // the blocks of the sink's extra range (none for GradSink)
    int xblocks = 0;
    if constexpr (Sink::kExtra) {
        const int64_t q = (sk.xn + 3) / 4;
        xblocks = sk.xn > 0 ? (int)((q + threads - 1) / threads < 64 ? (q + threads - 1) / threads : 64) : 0;
    }
    const int blocks = gblocks + xblocks;
#define LE_PREB(DEG)                                                                                               \
    preprocess_bwd_kernel<DEG, Sink><<<blocks, threads, 0, s>>>(g->n, g->means, g->log_scales, g->quats,           \
                                                                g->opacity_raw, g->sh, cp, pr->tiles_touched,      \
                                                                pr->clamp_mask,                                    \
                                                                reinterpret_cast<const float4*>(grad2d), sk)
    switch (g->sh_degree) {
        case 0: LE_PREB(0); break;
        case 1: LE_PREB(1); break;
        case 2: LE_PREB(2); break;
        default: LE_PREB(3); break;
    }
#undef LE_PREB
    LE_LAUNCHED();
    return LE_OK;
}

le_status preprocess_backward(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                              const float* grad2d, const le_gaussian_grads* out, cudaStream_t s)
{
    const GradSink sk{{out->means, out->log_scales, out->quats, out->opacity_raw, out->sh, out->feat, out->unc}};
    return launch_preprocess_backward(cam, g, pr, grad2d, sk, s);
}

le_status preprocess_backward_adam(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                                   const float* grad2d, const le_gaussian_grads* m, const le_gaussian_grads* v,
                                   const AdamParams& h, cudaStream_t s, float* xp, const float* xg, float* xm,
                                   float* xv, int64_t xn)
{
    AdamSink sk;
    sk.xp = xp;
    sk.xg = xg;
    sk.xm = xm;
    sk.xv = xv;
    sk.xn = xn;
    sk.gblocks = (g->n + 127) / 128;
    float* const p[7] = {const_cast<float*>(g->means), const_cast<float*>(g->log_scales), const_cast<float*>(g->quats),
                         const_cast<float*>(g->opacity_raw), const_cast<float*>(g->sh), const_cast<float*>(g->feat),
                         const_cast<float*>(g->unc)};
    float* const mm[7] = {m->means, m->log_scales, m->quats, m->opacity_raw, m->sh, m->feat, m->unc};
    float* const vv[7] = {v->means, v->log_scales, v->quats, v->opacity_raw, v->sh, v->feat, v->unc};
    for (int f = 0; f < 7; ++f) {
        sk.p[f] = p[f];
        sk.m[f] = mm[f];
        sk.v[f] = vv[f];
    }
    sk.h = h;
    return launch_preprocess_backward(cam, g, pr, grad2d, sk, s);
}
}  // namespace leg
