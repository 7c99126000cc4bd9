// Training helpers of Sec. 4: the RGB L1 term and a fused Adam update over a
// flat parameter buffer (lr 1e-3, betas (0.9, 0.999) in the paper).
#include "common.cuh"

namespace leg {
namespace {

__global__ void __launch_bounds__(256) l1_kernel(int64_t n, const float* __restrict__ img,
                                                 const float* __restrict__ target, float* __restrict__ loss,
                                                 float* __restrict__ grad, float inv_n)
{
    float s = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float r = img[i] - target[i];
        s += fabsf(r);
        grad[i] = (r > 0.f ? inv_n : (r < 0.f ? -inv_n : 0.f));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += ws[w];
        atomicAdd(loss, t * inv_n);
    }
}

// float4 body over the first n/4 quads; the n % 4 tail elements scalar.
__global__ void __launch_bounds__(256) adam_kernel(int64_t n, float* __restrict__ p, const float* __restrict__ g,
                                                   float* __restrict__ m, float* __restrict__ v, AdamParams h,
                                                   float lo, float hi)
{
    const int64_t n4 = n / 4;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n4; i += stride) {
        float4 pp = reinterpret_cast<float4*>(p)[i], mm = reinterpret_cast<float4*>(m)[i];
        float4 vv = reinterpret_cast<float4*>(v)[i];
        const float4 gg = reinterpret_cast<const float4*>(g)[i];
        adam_step4(pp, gg, mm, vv, h, lo, hi);
        reinterpret_cast<float4*>(p)[i] = pp;
        reinterpret_cast<float4*>(m)[i] = mm;
        reinterpret_cast<float4*>(v)[i] = vv;
    }
    const int64_t t = 4 * n4 + tid;
    if (t < n) p[t] = adam_step(p[t], g[t], m[t], v[t], h, lo, hi);
}

}  // namespace

AdamParams adam_params(int32_t step, float lr, float beta1, float beta2, float eps)
{
    const double c1 = 1.0 - pow((double)beta1, step), c2 = 1.0 - pow((double)beta2, step);
    return AdamParams{beta1, beta2, 1.0f - beta1, 1.0f - beta2, (float)(lr / c1), (float)(1.0 / sqrt(c2)), eps};
}

}  // namespace leg

using namespace leg;

extern "C" le_status le_rgb_l1(int64_t n, const float* img, const float* target, float* loss, float* grad,
                               void* stream)
{
    LE_TRACE("le_rgb_l1");
    LE_CHECK_ARG(n >= 0, "n < 0");
    if (n == 0) return LE_OK;
    LE_CHECK_ARG(img && target && loss && grad, "null pointer");
    const int blocks = (int)((n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8);
    LE_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), as_stream(stream)));
    l1_kernel<<<blocks, 256, 0, as_stream(stream)>>>(n, img, target, loss, grad, 1.0f / (float)n);
    LE_LAUNCHED();
    return LE_OK;
}

extern "C" le_status le_adam(int64_t n, float* param, const float* grad, float* m, float* v, int32_t step, float lr,
                             float beta1, float beta2, float eps, float clamp_lo, float clamp_hi, void* stream)
{
    LE_TRACE("le_adam");
    LE_CHECK_ARG(n >= 0 && step >= 1, "n < 0 or step < 1");
    if (n == 0) return LE_OK;
    LE_CHECK_ARG(param && grad && m && v, "null pointer");
    LE_CHECK_ARG(aligned16(param) && aligned16(grad) && aligned16(m) && aligned16(v),
                 "Adam buffers must be 16-byte aligned");
    const int64_t n4 = n / 4 + 1;
    const int blocks = (int)((n4 + 255) / 256 < 152 * 16 ? (n4 + 255) / 256 : 152 * 16);
    adam_kernel<<<blocks, 256, 0, as_stream(stream)>>>(n, param, grad, m, v,
                                                        adam_params(step, lr, beta1, beta2, eps), clamp_lo, clamp_hi);
    LE_LAUNCHED();
    return LE_OK;
}
