// Open-vocabulary relevancy (supp. Sec. "Inference"): F = M_infer S, then the
// LERF relevancy of F's CLIP part against text prompts and canonical
// negatives.  Reading of that relevancy: phi = F_clip / |F_clip|,
// rel_j = min_k e^{phi.q_j} / (e^{phi.q_j} + e^{phi.n_k}) = 1/(1 + e^{max_k phi.n_k - phi.q_j}).
//
// Unfused FP32 path: F is materialised in chunks of pixels through the
// workspace by a CUDA-core GEMM, then one thread per pixel reduces it.
#include "common.cuh"
#include "gemm_fp32.cuh"

namespace leg {

le_status query_fused(int32_t P, const float* feat, const le_decoder* dec, const float* codebook, int32_t d,
                      int32_t d_clip, const float* text, int32_t Q, const float* negs, int32_t n_neg, float* rel,
                      void* ws, size_t ws_bytes, cudaStream_t s);
size_t query_fused_workspace(int32_t P, int32_t n_cb, int32_t d_clip);
le_status check_decoder(const le_decoder* d);

namespace {

constexpr int kChunk = 65536;
constexpr int kMaxEmb = 16;

// One thread per pixel of the chunk: |F_clip|, dots with the text and negative
// embeddings (staged in shared memory), relevancy.
__global__ void __launch_bounds__(256) relevancy_kernel(int n, int d_clip, const float* __restrict__ F,
                                                        const float* __restrict__ text, int Q,
                                                        const float* __restrict__ negs, int n_neg,
                                                        float* __restrict__ rel, int64_t rel_stride)
{
    extern __shared__ float emb[];     // [(Q + n_neg)][d_clip]
    const int ne = Q + n_neg;
    for (int i = threadIdx.x; i < ne * d_clip; i += blockDim.x)
        emb[i] = i < Q * d_clip ? text[i] : negs[i - Q * d_clip];
    __syncthreads();
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float dots[kMaxEmb];
#pragma unroll
    for (int j = 0; j < kMaxEmb; ++j) dots[j] = 0.f;
    float n2 = 0.f;
    for (int e = 0; e < d_clip; ++e) {
        const float f = F[(size_t)e * n + p];
        n2 = fmaf(f, f, n2);
#pragma unroll
        for (int j = 0; j < kMaxEmb; ++j)
            if (j < ne) dots[j] = fmaf(f, emb[j * d_clip + e], dots[j]);
    }
    const float inv = rsqrtf(n2);
    float smax = -INFINITY;
#pragma unroll
    for (int j = 0; j < kMaxEmb; ++j)
        if (j >= Q && j < ne) smax = fmaxf(smax, dots[j] * inv);
#pragma unroll
    for (int j = 0; j < kMaxEmb; ++j)
        if (j < Q) rel[(size_t)j * rel_stride + p] = 1.f / (1.f + expf(smax - dots[j] * inv));
}

}  // namespace
}  // namespace leg

using namespace leg;

extern "C" le_status le_query_workspace(int32_t mode, int32_t P, int32_t n_cb, int32_t d_clip, size_t* bytes)
{
    LE_TRACE("le_query_workspace");
    LE_CHECK_ARG(bytes && P >= 0 && n_cb > 0 && d_clip > 0, "bad arguments");
    if (mode == LE_DECODE_FUSED_BF16) {
        *bytes = query_fused_workspace(P, n_cb, d_clip);
        return LE_OK;
    }
    LE_CHECK_ARG(mode == LE_DECODE_UNFUSED_FP32, "unknown mode %d", mode);
    const int chunk = P < kChunk ? P : kChunk;
    *bytes = sizeof(float) * (size_t)d_clip * (chunk > 0 ? chunk : 1);
    return LE_OK;
}

extern "C" le_status le_query(int32_t mode, int32_t P, const float* feat, const le_decoder* dec, const float* prob,
                              const float* codebook, int32_t d, int32_t d_clip, const float* text, int32_t Q,
                              const float* negs, int32_t n_neg, float* relevancy, void* workspace,
                              size_t workspace_bytes, void* stream)
{
    LE_TRACE("le_query");
    LE_CHECK_ARG(P >= 0 && d > 0 && d_clip > 0 && d_clip <= d, "bad sizes");
    LE_CHECK_ARG(Q >= 1 && n_neg >= 1 && Q + n_neg <= kMaxEmb, "need 1 <= Q, n_neg and Q + n_neg <= %d", kMaxEmb);
    LE_CHECK_ARG(codebook && text && negs && (P == 0 || relevancy), "null pointer");
    if (P == 0) return LE_OK;
    cudaStream_t s = as_stream(stream);
    size_t need = 0;
    le_status st;
    if (mode == LE_DECODE_FUSED_BF16) {
        if ((st = check_decoder(dec)) != LE_OK) return st;
        LE_CHECK_ARG(feat != nullptr, "fused query needs feat");
        need = query_fused_workspace(P, dec->n_cb, d_clip);
        LE_CHECK_ARG(workspace_bytes >= need && (need == 0 || workspace), "workspace too small");
        return query_fused(P, feat, dec, codebook, d, d_clip, text, Q, negs, n_neg, relevancy, workspace,
                           workspace_bytes, s);
    }
    LE_CHECK_ARG(mode == LE_DECODE_UNFUSED_FP32, "unknown mode %d", mode);
    LE_CHECK_ARG(prob != nullptr, "unfused query needs prob");
    if ((st = le_query_workspace(mode, P, 1, d_clip, &need)) != LE_OK) return st;
    LE_CHECK_ARG(workspace && workspace_bytes >= need, "workspace too small: %zu < %zu", workspace_bytes, need);
    // n_cb is implied by the codebook pointer contract: prob is [n_cb, P], codebook [n_cb, d]
    const int n_cb = dec ? dec->n_cb : 0;
    LE_CHECK_ARG(n_cb > 0, "unfused query needs dec->n_cb for the codebook size");
    float* F = static_cast<float*>(workspace);
    const int ne = Q + n_neg;
    const size_t smem = sizeof(float) * ne * d_clip;
    LE_CHECK_ARG(smem <= 200 * 1024, "too many embeddings for shared memory");
    if (smem > 48 * 1024)
        LE_CUDA(cudaFuncSetAttribute(relevancy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int p0 = 0; p0 < P; p0 += kChunk) {
        const int n = P - p0 < kChunk ? P - p0 : kChunk;
        GemmArgs g{};
        g.M = d_clip; g.N = n; g.K = n_cb;
        g.A = codebook; g.lda = d;         // A(e, i) = S[i][e]
        g.B = prob + p0; g.ldb = P;        // B(i, p) = prob[i][p0 + p]
        g.C = F; g.ldc = n;
        if ((st = sgemm(true, false, g, 1, s)) != LE_OK) return st;
        relevancy_kernel<<<(n + 255) / 256, 256, smem, s>>>(n, d_clip, F, text, Q, negs, n_neg, relevancy + p0, P);
        LE_LAUNCHED();
    }
    return LE_OK;
}
