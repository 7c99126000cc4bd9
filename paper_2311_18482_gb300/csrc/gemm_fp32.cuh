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

// (64 MI) x (64 NJ) output tile per block of 256 threads (MI, NJ in {1, 2}), K
// in steps of 8 through double-buffered shared memory (the next step's
// elements are loaded into registers while the current step is multiplied).
// Thread (tx, ty) owns rows {4ty..4ty+3} (and 64+4ty.. when MI = 2) and the
// same columns in tx: MI x NJ blocks of 4 x 4, read from shared memory as
// float4 without bank conflicts.
constexpr int kGK = 8;

template <int MI, int NJ, bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_kernel(GemmArgs a)
{
    constexpr int BM = 64 * MI, BN = 64 * NJ, LA = BM * kGK / 256, LB = BN * kGK / 256;
    __shared__ __align__(16) float As[2][kGK][BM];
    __shared__ __align__(16) float Bs[2][kGK][BN];
    const int bm = blockIdx.y * BM, bn = blockIdx.x * BN;
    const int kchunk = ((a.K + gridDim.z - 1) / gridDim.z + kGK - 1) / kGK * kGK;
    const int k0 = blockIdx.z * kchunk, k1 = min(a.K, k0 + kchunk);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float ra[LA], rb[LB];
    // element l of this thread's share of the (kk) step: A(m, k) and B(k, n)
    auto load = [&](int kk) {
#pragma unroll
        for (int l = 0; l < LA; ++l) {
            const int idx = threadIdx.x + l * 256;
            int m, k;
            if (!TA) { m = idx / kGK; k = idx % kGK; } else { k = idx / BM; m = idx % BM; }
            const int gm = bm + m, gk = kk + k;
            ra[l] = gm < a.M && gk < k1 ? (TA ? a.A[(size_t)gk * a.lda + gm] : a.A[(size_t)gm * a.lda + gk]) : 0.f;
        }
#pragma unroll
        for (int l = 0; l < LB; ++l) {
            const int idx = threadIdx.x + l * 256;
            int n, k2;
            if (!TB) { k2 = idx / BN; n = idx % BN; } else { n = idx / kGK; k2 = idx % kGK; }
            const int gn = bn + n, gk2 = kk + k2;
            rb[l] = gn < a.N && gk2 < k1 ? (TB ? a.B[(size_t)gn * a.ldb + gk2] : a.B[(size_t)gk2 * a.ldb + gn]) : 0.f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int l = 0; l < LA; ++l) {
            const int idx = threadIdx.x + l * 256;
            int m, k;
            if (!TA) { m = idx / kGK; k = idx % kGK; } else { k = idx / BM; m = idx % BM; }
            As[buf][k][m] = ra[l];
        }
#pragma unroll
        for (int l = 0; l < LB; ++l) {
            const int idx = threadIdx.x + l * 256;
            int n, k2;
            if (!TB) { k2 = idx / BN; n = idx % BN; } else { n = idx / kGK; k2 = idx % kGK; }
            Bs[buf][k2][n] = rb[l];
        }
    };
    float acc[4 * MI][4 * NJ] = {};
    if (k0 < k1) {
        load(k0);
        store(0);
    }
    __syncthreads();
    int buf = 0;
    for (int kk = k0; kk < k1; kk += kGK) {
        const bool more = kk + kGK < k1;
        if (more) load(kk + kGK);
#pragma unroll
        for (int k = 0; k < kGK; ++k) {
            float av[4 * MI], bv[4 * NJ];
#pragma unroll
            for (int h = 0; h < MI; ++h) {
                const float4 x = *reinterpret_cast<const float4*>(&As[buf][k][64 * h + 4 * ty]);
                av[4 * h] = x.x; av[4 * h + 1] = x.y; av[4 * h + 2] = x.z; av[4 * h + 3] = x.w;
            }
#pragma unroll
            for (int h = 0; h < NJ; ++h) {
                const float4 x = *reinterpret_cast<const float4*>(&Bs[buf][k][64 * h + 4 * tx]);
                bv[4 * h] = x.x; bv[4 * h + 1] = x.y; bv[4 * h + 2] = x.z; bv[4 * h + 3] = x.w;
            }
#pragma unroll
            for (int i = 0; i < 4 * MI; ++i)
#pragma unroll
                for (int j = 0; j < 4 * NJ; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 4 * MI; ++i) {
        const int m = bm + 64 * (i >> 2) + 4 * ty + (i & 3);
        if (m >= a.M) continue;
#pragma unroll
        for (int j = 0; j < 4 * NJ; ++j) {
            const int n = bn + 64 * (j >> 2) + 4 * tx + (j & 3);
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

template <bool TA, bool TB>
void sgemm_launch(const GemmArgs& a, int ksplit, cudaStream_t s)
{
    const int z = ksplit > 0 ? ksplit : 1;
    const bool wm = a.M > 64, wn = a.N > 64;
    const dim3 grid((a.N + (wn ? 127 : 63)) / (wn ? 128 : 64), (a.M + (wm ? 127 : 63)) / (wm ? 128 : 64), z);
    if (wm && wn) sgemm_kernel<2, 2, TA, TB><<<grid, 256, 0, s>>>(a);
    else if (wn) sgemm_kernel<1, 2, TA, TB><<<grid, 256, 0, s>>>(a);
    else if (wm) sgemm_kernel<2, 1, TA, TB><<<grid, 256, 0, s>>>(a);
    else sgemm_kernel<1, 1, TA, TB><<<grid, 256, 0, s>>>(a);
}

// One launch: each side of the output tile 128 where that side of C exceeds 64,
// else 64; ksplit > 1 splits K over gridDim.z (with a.atomic set).
inline le_status sgemm(bool ta, bool tb, const GemmArgs& a, int ksplit, cudaStream_t s)
{
    if (!ta && !tb) sgemm_launch<false, false>(a, ksplit, s);
    else if (ta && !tb) sgemm_launch<true, false>(a, ksplit, s);
    else if (!ta && tb) sgemm_launch<false, true>(a, ksplit, s);
    else sgemm_launch<true, true>(a, ksplit, s);
    LE_LAUNCHED();
    return LE_OK;
}

}  // namespace leg
