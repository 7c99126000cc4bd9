// RGB reconstruction loss of 3D Gaussian Splatting, which Sec. 4 keeps:
//   L = (1 - lambda) L1 + lambda (1 - SSIM),  lambda = 0.2,
// SSIM per channel with an 11 x 11 Gaussian window (sigma 1.5), zero padding,
// C1 = 0.01^2, C2 = 0.03^2, averaged over pixels and channels.
//
// ssim_fwd_kernel: one 16 x 16 tile per block, per channel: the 26 x 26 input
// window (tile + 5-pixel halo, zero outside the image) into shared memory,
// a horizontal 11-tap pass of the five statistics (x, y, x^2, y^2, x y), a
// vertical pass; per pixel S and the three partial-derivative maps
//   A = dS/dmu_x - 2 mu_x dS/dsigma_x^2 - mu_y dS/dsigma_xy, B = dS/dsigma_x^2, C = dS/dsigma_xy,
// block sums of S and |x - y|.
// ssim_bwd_kernel: the same two-pass blur of A, B, C; the gradient
//   dL/dx = ((1 - lambda) sign(x - y) - lambda (G*A + 2 x G*B + y G*C)) / (3 P).
#include "common.cuh"

namespace leg {
namespace {

constexpr int kT = 16, kR = 5, kWin = kT + 2 * kR;   // tile, halo, window edge (26)

struct SsimParams {
    int W, H;
    float w[2 * kR + 1];        // normalised 1-D Gaussian window
    float lambda, inv3P;
};

__device__ __forceinline__ float block_sum(float v, float* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kT * kT) ssim_fwd_kernel(SsimParams sp, const float* __restrict__ img,
                                                           const float* __restrict__ tgt, float* __restrict__ maps,
                                                           float* __restrict__ acc)
{
    __shared__ float sx[kWin][kWin + 1], sy[kWin][kWin + 1];
    __shared__ float hb[5][kWin][kT + 1];
    __shared__ float red[8];
    const int x0 = blockIdx.x * kT - kR, y0 = blockIdx.y * kT - kR;
    const int tx = threadIdx.x & (kT - 1), ty = threadIdx.x / kT;
    const int px = blockIdx.x * kT + tx, py = blockIdx.y * kT + ty;
    const bool inside = px < sp.W && py < sp.H;
    const size_t P = (size_t)sp.W * sp.H;
    const float C1 = 0.01f * 0.01f, C2 = 0.03f * 0.03f;
    float ssum = 0.f, l1 = 0.f;
    for (int c = 0; c < 3; ++c) {
        const float* X = img + c * P;
        const float* Y = tgt + c * P;
        for (int i = threadIdx.x; i < kWin * kWin; i += blockDim.x) {
            const int r = i / kWin, q = i % kWin, gy = y0 + r, gx = x0 + q;
            const bool in = gx >= 0 && gx < sp.W && gy >= 0 && gy < sp.H;
            sx[r][q] = in ? X[(size_t)gy * sp.W + gx] : 0.f;
            sy[r][q] = in ? Y[(size_t)gy * sp.W + gx] : 0.f;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kWin * kT; i += blockDim.x) {
            const int r = i / kT, q = i % kT;
            float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int b = 0; b <= 2 * kR; ++b) {
                const float a = sx[r][q + b], d = sy[r][q + b], w = sp.w[b];
                m[0] = fmaf(w, a, m[0]);
                m[1] = fmaf(w, d, m[1]);
                m[2] = fmaf(w, a * a, m[2]);
                m[3] = fmaf(w, d * d, m[3]);
                m[4] = fmaf(w, a * d, m[4]);
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) hb[k][r][q] = m[k];
        }
        __syncthreads();
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a <= 2 * kR; ++a)
#pragma unroll
            for (int k = 0; k < 5; ++k) m[k] = fmaf(sp.w[a], hb[k][ty + a][tx], m[k]);
        const float mx = m[0], my = m[1];
        const float vx = m[2] - mx * mx, vy = m[3] - my * my, cxy = m[4] - mx * my;
        const float n1 = 2.f * mx * my + C1, n2 = 2.f * cxy + C2;
        const float d1 = mx * mx + my * my + C1, d2 = vx + vy + C2;
        const float inv12 = 1.f / (d1 * d2);
        const float S = n1 * n2 * inv12;
        const float dmu = 2.f * my * n2 * inv12 - 2.f * mx * S / d1;
        const float dvx = -S / d2;
        const float dcxy = 2.f * n1 * inv12;
        if (inside) {
            const size_t o = (size_t)py * sp.W + px;
            maps[(3 * c) * P + o] = dmu - 2.f * mx * dvx - my * dcxy;
            maps[(3 * c + 1) * P + o] = dvx;
            maps[(3 * c + 2) * P + o] = dcxy;
            ssum += S;
            l1 += fabsf(sx[ty + kR][tx + kR] - sy[ty + kR][tx + kR]);
        }
        __syncthreads();
    }
    const float s1 = block_sum(ssum, red);
    const float s2 = block_sum(l1, red);
    if (threadIdx.x == 0) {
        atomicAdd(acc, s2);
        atomicAdd(acc + 1, s1);
    }
}

__global__ void __launch_bounds__(kT * kT) ssim_bwd_kernel(SsimParams sp, const float* __restrict__ img,
                                                           const float* __restrict__ tgt,
                                                           const float* __restrict__ maps, float* __restrict__ grad)
{
    __shared__ float sm[3][kWin][kWin + 1];
    __shared__ float hb[3][kWin][kT + 1];
    const int x0 = blockIdx.x * kT - kR, y0 = blockIdx.y * kT - kR;
    const int tx = threadIdx.x & (kT - 1), ty = threadIdx.x / kT;
    const int px = blockIdx.x * kT + tx, py = blockIdx.y * kT + ty;
    const bool inside = px < sp.W && py < sp.H;
    const size_t P = (size_t)sp.W * sp.H;
    for (int c = 0; c < 3; ++c) {
        for (int i = threadIdx.x; i < kWin * kWin; i += blockDim.x) {
            const int r = i / kWin, q = i % kWin, gy = y0 + r, gx = x0 + q;
            const bool in = gx >= 0 && gx < sp.W && gy >= 0 && gy < sp.H;
            const size_t o = (size_t)gy * sp.W + gx;
#pragma unroll
            for (int k = 0; k < 3; ++k) sm[k][r][q] = in ? maps[(3 * c + k) * P + o] : 0.f;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kWin * kT; i += blockDim.x) {
            const int r = i / kT, q = i % kT;
            float m[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int b = 0; b <= 2 * kR; ++b)
#pragma unroll
                for (int k = 0; k < 3; ++k) m[k] = fmaf(sp.w[b], sm[k][r][q + b], m[k]);
#pragma unroll
            for (int k = 0; k < 3; ++k) hb[k][r][q] = m[k];
        }
        __syncthreads();
        float g[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a <= 2 * kR; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) g[k] = fmaf(sp.w[a], hb[k][ty + a][tx], g[k]);
        if (inside) {
            const size_t o = (size_t)py * sp.W + px;
            const float x = img[c * P + o], y = tgt[c * P + o];
            const float s1 = x > y ? 1.f : (x < y ? -1.f : 0.f);
            const float dS = g[0] + 2.f * x * g[1] + y * g[2];
            grad[c * P + o] = ((1.f - sp.lambda) * s1 - sp.lambda * dS) * sp.inv3P;
        }
        __syncthreads();
    }
}

__global__ void rgb_loss_finalize_kernel(const float* __restrict__ acc, float inv3P, float lambda,
                                         float* __restrict__ loss)
{
    const float l1 = acc[0] * inv3P, ssim = acc[1] * inv3P;
    loss[0] = (1.f - lambda) * l1 + lambda * (1.f - ssim);
    loss[1] = l1;
    loss[2] = ssim;
}

}  // namespace
}  // namespace leg

using namespace leg;

extern "C" le_status le_rgb_loss_workspace(int32_t W, int32_t H, size_t* bytes)
{
    LE_TRACE("le_rgb_loss_workspace");
    LE_CHECK_ARG(bytes != nullptr, "bytes is null");
    LE_CHECK_ARG(W > 0 && H > 0, "bad image size");
    *bytes = ((size_t)9 * W * H + 64) * sizeof(float);
    return LE_OK;
}

extern "C" le_status le_rgb_loss(int32_t W, int32_t H, const float* img, const float* target, float lambda_ssim,
                                 float* loss, float* grad, void* workspace, size_t workspace_bytes, void* stream)
{
    LE_TRACE("le_rgb_loss");
    LE_CHECK_ARG(W > 0 && H > 0 && W <= 16384 && H <= 16384, "bad image size %d x %d", W, H);
    LE_CHECK_ARG(img && target && loss && grad && workspace, "null pointer");
    LE_CHECK_ARG(lambda_ssim >= 0.f && lambda_ssim <= 1.f, "lambda_ssim must be in [0, 1]");
    LE_CHECK_ARG(workspace_bytes >= ((size_t)9 * W * H + 64) * sizeof(float), "workspace too small");
    cudaStream_t s = as_stream(stream);
    float* maps = static_cast<float*>(workspace);
    float* acc = maps + (size_t)9 * W * H;
    LE_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(float), s));
    SsimParams sp;
    sp.W = W;
    sp.H = H;
    double g[2 * 5 + 1], tot = 0.0;
    for (int k = -5; k <= 5; ++k) tot += (g[k + 5] = exp(-(double)(k * k) / (2.0 * 1.5 * 1.5)));
    for (int k = 0; k <= 10; ++k) sp.w[k] = (float)(g[k] / tot);
    sp.lambda = lambda_ssim;
    sp.inv3P = (float)(1.0 / (3.0 * (double)W * H));
    const dim3 grid((W + 15) / 16, (H + 15) / 16);
    ssim_fwd_kernel<<<grid, 256, 0, s>>>(sp, img, target, maps, acc);
    LE_LAUNCHED();
    ssim_bwd_kernel<<<grid, 256, 0, s>>>(sp, img, target, maps, grad);
    LE_LAUNCHED();
    rgb_loss_finalize_kernel<<<1, 1, 0, s>>>(acc, sp.inv3P, lambda_ssim, loss);
    LE_LAUNCHED();
    return LE_OK;
}
