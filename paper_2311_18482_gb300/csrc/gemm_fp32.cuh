// Plain FP32 tiled GEMM on CUDA cores, used by the unfused decoder and query
// paths (their "plain FP32" reference form):
//   C[m][n] = epilogue( sum_k A(m,k) B(k,n) )
//   A(m,k) = TA ? A[k*lda + m] : A[m*lda + k]      B(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n]
// epilogue: + bias[m], ReLU, mask (keep where mask[m*ldm+n] > 0), then store
// or atomically add (split over K with gridDim.z > 1).
#pragma once
#include "common.cuh"

namespace leg {

struct GemmArgs {
    int M, N, K;
    const float* A;
    int lda;
    const float* B;
    int ldb;
    float* C;
    int ldc;
    const float* bias;
    bool relu;
    const float* mask;
    int ldm;
    bool atomic;
};

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_kernel(GemmArgs a)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int bm = blockIdx.y * BM, bn = blockIdx.x * BN;
    const int kchunk = ((a.K + gridDim.z - 1) / gridDim.z + BK - 1) / BK * BK;
    const int k0 = blockIdx.z * kchunk, k1 = min(a.K, k0 + kchunk);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int kk = k0; kk < k1; kk += BK) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int idx = threadIdx.x + l * 256;
            int m, k;
            if (!TA) { k = idx % BK; m = idx / BK; }
            else { m = idx % BM; k = idx / BM; }
            const int gm = bm + m, gk = kk + k;
            float v = 0.f;
            if (gm < a.M && gk < k1) v = TA ? a.A[(size_t)gk * a.lda + gm] : a.A[(size_t)gm * a.lda + gk];
            As[k][m] = v;
            int n, k2;
            if (!TB) { n = idx % BN; k2 = idx / BN; }
            else { k2 = idx % BK; n = idx / BK; }
            const int gn = bn + n, gk2 = kk + k2;
            float w = 0.f;
            if (gn < a.N && gk2 < k1) w = TB ? a.B[(size_t)gn * a.ldb + gk2] : a.B[(size_t)gk2 * a.ldb + gn];
            Bs[k2][n] = w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            float av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[k][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[k][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = bm + ty * 4 + i;
        if (m >= a.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = bn + tx * 4 + j;
            if (n >= a.N) continue;
            float v = acc[i][j];
            if (a.bias) v += a.bias[m];
            if (a.relu) v = fmaxf(v, 0.f);
            if (a.mask && !(a.mask[(size_t)m * a.ldm + n] > 0.f)) v = 0.f;
            float* c = a.C + (size_t)m * a.ldc + n;
            if (a.atomic) atomicAdd(c, v);
            else *c = v;
        }
    }
}

inline le_status sgemm(bool ta, bool tb, const GemmArgs& a, int ksplit, cudaStream_t s)
{
    dim3 grid((a.N + 63) / 64, (a.M + 63) / 64, ksplit > 0 ? ksplit : 1);
    if (!ta && !tb) sgemm_kernel<false, false><<<grid, 256, 0, s>>>(a);
    else if (ta && !tb) sgemm_kernel<true, false><<<grid, 256, 0, s>>>(a);
    else if (!ta && tb) sgemm_kernel<false, true><<<grid, 256, 0, s>>>(a);
    else sgemm_kernel<true, true><<<grid, 256, 0, s>>>(a);
    LE_LAUNCHED();
    return LE_OK;
}

}  // namespace leg
