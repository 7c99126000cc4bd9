// Semantic decoder D_MLP (Eq. 8, eq:lem_dec; supp. Tab. dmlp), softmax,
// uncertainty-weighted cross-entropy (Eqs. 9-12) and its backward pass --
// the unfused FP32 path: every layer is a CUDA-core GEMM over all pixels whose
// activations and logits go through HBM (workspace).  It is the fallback of
// the fused tcgen05 path (decoder_tc.cu) and the reference its error is measured
// against.  le_decode dispatches between the two.
#include "common.cuh"
#include "gemm_fp32.cuh"

namespace leg {

le_status decode_fused(int32_t P, const float* feat, const float* unc, const le_decoder* dec, const int32_t* target,
                       float lambda_ce, float lambda_u, float* loss, float* d_feat, float* d_unc,
                       const le_decoder_grads* dg, int32_t* argmax, float* prob, void* ws, size_t ws_bytes,
                       cudaStream_t s, const float* img = nullptr, const float* img_t = nullptr,
                       float* loss_l1 = nullptr, float* d_img = nullptr);
size_t decode_fused_workspace(int32_t P, const le_decoder* dec);
le_status check_fused_decoder(const le_decoder* dec, bool train);
bool wide_decoder(const le_decoder* d);
le_status check_wide_decoder(const le_decoder* d, bool train);
size_t wide_workspace(int32_t P, const le_decoder* d, bool train);
le_status wide_decode(int32_t P, const float* feat, const float* unc, const le_decoder* d, const int32_t* target,
                      float lambda_ce, float lambda_u, float* loss, float* d_feat, float* d_unc,
                      const le_decoder_grads* dg, int32_t* argmax, float* prob, void* ws, size_t ws_bytes,
                      cudaStream_t s);

namespace {

// Per pixel: max/argmax, log-sum-exp, then (training) CE, dz and dL/du, or
// (inference) the softmax.  Logits are planar [n_cb][P].
__global__ void __launch_bounds__(256) softmax_ce_kernel(int P, int ncb, const float* __restrict__ z,
                                                         const float* __restrict__ unc,
                                                         const int32_t* __restrict__ target, float lambda_ce,
                                                         float lambda_u, float* __restrict__ dz,
                                                         float* __restrict__ d_unc, float* __restrict__ loss,
                                                         int32_t* __restrict__ argmax, float* __restrict__ prob)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    float lce = 0.f, lu = 0.f;
    if (p < P) {
        float m = z[p];
        int am = 0;
        for (int c = 1; c < ncb; ++c) {
            const float v = z[(size_t)c * P + p];
            if (v > m) {
                m = v;
                am = c;
            }
        }
        float s = 0.f;
        for (int c = 0; c < ncb; ++c) s += expf(z[(size_t)c * P + p] - m);
        const float lse = m + logf(s);
        if (argmax) argmax[p] = am;
        if (prob)
            for (int c = 0; c < ncb; ++c) prob[(size_t)c * P + p] = expf(z[(size_t)c * P + p] - lse);
        if (target) {
            const int t = target[p];
            const float ce = lse - z[(size_t)t * P + p];
            const float u = unc[p];
            const float w = lambda_ce * (1.f - u) / (float)P;
            for (int c = 0; c < ncb; ++c)
                dz[(size_t)c * P + p] = w * (expf(z[(size_t)c * P + p] - lse) - (c == t ? 1.f : 0.f));
            d_unc[p] = (lambda_u - lambda_ce * ce) / (float)P;
            lce = ce * (1.f - u);
            lu = u;
        }
    }
    if (!target) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lce += __shfl_xor_sync(0xffffffffu, lce, o);
        lu += __shfl_xor_sync(0xffffffffu, lu, o);
    }
    __shared__ float ws[2][8];
    if ((threadIdx.x & 31) == 0) {
        ws[0][threadIdx.x >> 5] = lce;
        ws[1][threadIdx.x >> 5] = lu;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < 8; ++w) {
            a += ws[0][w];
            b += ws[1][w];
        }
        atomicAdd(loss, a / (float)P);
        atomicAdd(loss + 1, b / (float)P);
    }
}

// out[m] += sum_n A[m*lda + n] over this block's column chunk.
__global__ void __launch_bounds__(256) rowsum_kernel(int N, const float* __restrict__ A, int lda,
                                                     float* __restrict__ out)
{
    const int m = blockIdx.y;
    const int chunk = (N + gridDim.x - 1) / gridDim.x;
    const int n0 = blockIdx.x * chunk, n1 = min(N, n0 + chunk);
    float s = 0.f;
    for (int n = n0 + threadIdx.x; n < n1; n += 256) s += A[(size_t)m * lda + n];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += ws[w];
        atomicAdd(out + m, t);
    }
}

struct UnfusedWs {
    float *h1, *h2, *z, *dz, *dh2, *dh1;
    size_t bytes;
};

UnfusedWs unfused_layout(char* base, int32_t P, const le_decoder* d)
{
    UnfusedWs w;
    size_t off = 0;
    auto take = [&](size_t n) {
        float* p = base ? reinterpret_cast<float*>(base + off) : nullptr;
        off = align_up(off + n * sizeof(float), 256);
        return p;
    };
    w.h1 = take((size_t)d->h1 * P);
    w.h2 = take((size_t)d->h2 * P);
    w.z = take((size_t)d->n_cb * P);
    w.dz = take((size_t)d->n_cb * P);
    w.dh2 = take((size_t)d->h2 * P);
    w.dh1 = take((size_t)d->h1 * P);
    w.bytes = off;
    return w;
}

GemmArgs gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc)
{
    GemmArgs g{};
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
    return g;
}

le_status decode_unfused(int32_t P, const float* feat, const float* unc, const le_decoder* d, const int32_t* target,
                         float lambda_ce, float lambda_u, float* loss, float* d_feat, float* d_unc,
                         const le_decoder_grads* dg, int32_t* argmax, float* prob, float* logits, void* ws,
                         cudaStream_t s)
{
    UnfusedWs w = unfused_layout(static_cast<char*>(ws), P, d);
    float* z = logits ? logits : w.z;
    le_status st;
    // forward: h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), z = W3 h2 + b3
    GemmArgs g = gemm(d->h1, P, d->d_in, d->W1, d->d_in, feat, P, w.h1, P);
    g.bias = d->b1;
    g.relu = true;
    if ((st = sgemm(false, false, g, 1, s)) != LE_OK) return st;
    g = gemm(d->h2, P, d->h1, d->W2, d->h1, w.h1, P, w.h2, P);
    g.bias = d->b2;
    g.relu = true;
    if ((st = sgemm(false, false, g, 1, s)) != LE_OK) return st;
    g = gemm(d->n_cb, P, d->h2, d->W3, d->h2, w.h2, P, z, P);
    g.bias = d->b3;
    if ((st = sgemm(false, false, g, 1, s)) != LE_OK) return st;
    if (target) LE_CUDA(cudaMemsetAsync(loss, 0, 2 * sizeof(float), s));
    softmax_ce_kernel<<<(P + 255) / 256, 256, 0, s>>>(P, d->n_cb, z, unc, target, lambda_ce, lambda_u, w.dz, d_unc,
                                                      loss, argmax, prob);
    LE_LAUNCHED();
    if (!target) return LE_OK;

    // weight gradients accumulate atomically over split-K chunks of pixels
    LE_CUDA(cudaMemsetAsync(dg->W1, 0, sizeof(float) * d->h1 * d->d_in, s));
    LE_CUDA(cudaMemsetAsync(dg->b1, 0, sizeof(float) * d->h1, s));
    LE_CUDA(cudaMemsetAsync(dg->W2, 0, sizeof(float) * d->h2 * d->h1, s));
    LE_CUDA(cudaMemsetAsync(dg->b2, 0, sizeof(float) * d->h2, s));
    LE_CUDA(cudaMemsetAsync(dg->W3, 0, sizeof(float) * d->n_cb * d->h2, s));
    LE_CUDA(cudaMemsetAsync(dg->b3, 0, sizeof(float) * d->n_cb, s));
    const int split = 152;
    // layer 3: dW3 = dz h2^T, db3 = rowsum dz, dh2 = (W3^T dz) * [h2 > 0]
    g = gemm(d->n_cb, d->h2, P, w.dz, P, w.h2, P, dg->W3, d->h2);
    g.atomic = true;
    if ((st = sgemm(false, true, g, split, s)) != LE_OK) return st;
    rowsum_kernel<<<dim3(64, d->n_cb), 256, 0, s>>>(P, w.dz, P, dg->b3);
    LE_LAUNCHED();
    g = gemm(d->h2, P, d->n_cb, d->W3, d->h2, w.dz, P, w.dh2, P);
    g.mask = w.h2;
    g.ldm = P;
    if ((st = sgemm(true, false, g, 1, s)) != LE_OK) return st;
    // layer 2
    g = gemm(d->h2, d->h1, P, w.dh2, P, w.h1, P, dg->W2, d->h1);
    g.atomic = true;
    if ((st = sgemm(false, true, g, split, s)) != LE_OK) return st;
    rowsum_kernel<<<dim3(64, d->h2), 256, 0, s>>>(P, w.dh2, P, dg->b2);
    LE_LAUNCHED();
    g = gemm(d->h1, P, d->h2, d->W2, d->h1, w.dh2, P, w.dh1, P);
    g.mask = w.h1;
    g.ldm = P;
    if ((st = sgemm(true, false, g, 1, s)) != LE_OK) return st;
    // layer 1
    g = gemm(d->h1, d->d_in, P, w.dh1, P, feat, P, dg->W1, d->d_in);
    g.atomic = true;
    if ((st = sgemm(false, true, g, split, s)) != LE_OK) return st;
    rowsum_kernel<<<dim3(64, d->h1), 256, 0, s>>>(P, w.dh1, P, dg->b1);
    LE_LAUNCHED();
    g = gemm(d->d_in, P, d->h1, d->W1, d->d_in, w.dh1, P, d_feat, P);
    return sgemm(true, false, g, 1, s);
}

}  // namespace

le_status check_decoder(const le_decoder* d)
{
    LE_CHECK_ARG(d != nullptr, "decoder is null");
    LE_CHECK_ARG(d->d_in == LE_DFEAT, "decoder input width must be %d", LE_DFEAT);
    LE_CHECK_ARG(d->h1 > 0 && d->h2 > 0 && d->n_cb > 0 && d->h1 <= 4096 && d->h2 <= 4096 && d->n_cb <= 65536,
                 "decoder widths out of range");
    LE_CHECK_ARG(d->W1 && d->b1 && d->W2 && d->b2 && d->W3 && d->b3, "null decoder weight");
    return LE_OK;
}

}  // namespace leg

using namespace leg;

extern "C" le_status le_decode_workspace(int32_t mode, int32_t P, const le_decoder* dec, size_t* bytes)
{
    LE_TRACE("le_decode_workspace");
    LE_CHECK_ARG(bytes && dec && P >= 0, "bad arguments");
    const bool train = (mode & LE_DECODE_TRAIN) != 0;
    mode &= ~LE_DECODE_TRAIN;
    if (mode == LE_DECODE_FUSED_BF16) {
        *bytes = wide_decoder(dec) ? wide_workspace(P, dec, train) : decode_fused_workspace(P, dec);
        return LE_OK;
    }
    LE_CHECK_ARG(mode == LE_DECODE_UNFUSED_FP32, "unknown decode mode %d", mode);
    *bytes = unfused_layout(nullptr, P, dec).bytes;
    return LE_OK;
}

extern "C" le_status le_decode(int32_t mode, int32_t P, const float* feat, const float* unc, const le_decoder* dec,
                               const int32_t* target, float lambda_ce, float lambda_u, float* loss, float* d_feat,
                               float* d_unc, const le_decoder_grads* dgrads, int32_t* argmax, float* prob,
                               float* logits, void* workspace, size_t workspace_bytes, void* stream)
{
    LE_TRACE("le_decode");
    le_status st = check_decoder(dec);
    if (st != LE_OK) return st;
    LE_CHECK_ARG(P >= 0, "P < 0");
    LE_CHECK_ARG(mode == LE_DECODE_UNFUSED_FP32 || mode == LE_DECODE_FUSED_BF16, "unknown decode mode %d", mode);
    if (P == 0) {
        // no pixels: a training call's loss and weight gradients are zero
        if (target != nullptr || loss != nullptr) {
            LE_CHECK_ARG(loss && dgrads && dgrads->W1 && dgrads->b1 && dgrads->W2 && dgrads->b2 && dgrads->W3 &&
                             dgrads->b3,
                         "training needs loss and dgrads");
            cudaStream_t s = as_stream(stream);
            float* const z[7] = {loss, dgrads->W1, dgrads->b1, dgrads->W2, dgrads->b2, dgrads->W3, dgrads->b3};
            const size_t n[7] = {2, (size_t)dec->h1 * dec->d_in, (size_t)dec->h1, (size_t)dec->h2 * dec->h1,
                                 (size_t)dec->h2, (size_t)dec->n_cb * dec->h2, (size_t)dec->n_cb};
            for (int i = 0; i < 7; ++i) LE_CUDA(cudaMemsetAsync(z[i], 0, n[i] * sizeof(float), s));
        }
        return LE_OK;
    }
    LE_CHECK_ARG(feat != nullptr, "feat is null");
    const bool train = target != nullptr;
    if (train) {
        LE_CHECK_ARG(unc && loss && d_feat && d_unc && dgrads, "training needs unc, loss, d_feat, d_unc, dgrads");
        LE_CHECK_ARG(dgrads->W1 && dgrads->b1 && dgrads->W2 && dgrads->b2 && dgrads->W3 && dgrads->b3,
                     "null decoder gradient pointer");
    }
    cudaStream_t s = as_stream(stream);
    if (mode == LE_DECODE_FUSED_BF16) {
        LE_CHECK_ARG(logits == nullptr, "the fused path never materialises logits");
        if (wide_decoder(dec))
            return wide_decode(P, feat, unc, dec, target, lambda_ce, lambda_u, loss, d_feat, d_unc, dgrads, argmax,
                               prob, workspace, workspace_bytes, s);
        if ((st = check_fused_decoder(dec, train)) != LE_OK) return st;
        LE_CHECK_ARG(workspace_bytes >= decode_fused_workspace(P, dec), "workspace too small");
        return decode_fused(P, feat, unc, dec, target, lambda_ce, lambda_u, loss, d_feat, d_unc, dgrads, argmax,
                            prob, workspace, workspace_bytes, s);
    }
    const size_t need = unfused_layout(nullptr, P, dec).bytes;
    LE_CHECK_ARG(workspace && workspace_bytes >= need, "workspace too small: %zu < %zu", workspace_bytes, need);
    LE_CHECK_ARG((reinterpret_cast<uintptr_t>(workspace) & 255u) == 0, "workspace must be 256-byte aligned");
    return decode_unfused(P, feat, unc, dec, target, lambda_ce, lambda_u, loss, d_feat, d_unc, dgrads, argmax, prob,
                          logits, workspace, s);
}

extern "C" le_status le_decode_l1(int32_t mode, int32_t P, const float* feat, const float* unc,
                                  const le_decoder* dec, const int32_t* target, float lambda_ce, float lambda_u,
                                  float* loss, float* d_feat, float* d_unc, const le_decoder_grads* dgrads,
                                  const float* img, const float* img_target, float* loss_l1, float* d_img,
                                  void* workspace, size_t workspace_bytes, void* stream)
{
    LE_TRACE("le_decode_l1");
    le_status st = check_decoder(dec);
    if (st != LE_OK) return st;
    LE_CHECK_ARG(P > 0, "P must be positive");
    LE_CHECK_ARG(target != nullptr, "le_decode_l1 is a training call: target is null");
    LE_CHECK_ARG(img && img_target && loss_l1 && d_img, "null L1 pointer");
    // the 8-64-128 tensor-core training kernel computes the L1 term in the same pass
    if (mode == LE_DECODE_FUSED_BF16 && !wide_decoder(dec) && check_fused_decoder(dec, true) == LE_OK) {
        LE_CHECK_ARG(feat && unc && loss && d_feat && d_unc && dgrads, "training needs unc, loss, d_feat, d_unc, dgrads");
        LE_CHECK_ARG(dgrads->W1 && dgrads->b1 && dgrads->W2 && dgrads->b2 && dgrads->W3 && dgrads->b3,
                     "null decoder gradient pointer");
        LE_CHECK_ARG(workspace_bytes >= decode_fused_workspace(P, dec), "workspace too small");
        return decode_fused(P, feat, unc, dec, target, lambda_ce, lambda_u, loss, d_feat, d_unc, dgrads, nullptr,
                            nullptr, workspace, workspace_bytes, as_stream(stream), img, img_target, loss_l1, d_img);
    }
    if ((st = le_rgb_l1(3 * (int64_t)P, img, img_target, loss_l1, d_img, stream)) != LE_OK) return st;
    return le_decode(mode, P, feat, unc, dec, target, lambda_ce, lambda_u, loss, d_feat, d_unc, dgrads, nullptr,
                     nullptr, nullptr, workspace, workspace_bytes, stream);
}
