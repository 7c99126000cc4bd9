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

// 128 x 128 output tile per block of 256 threads, K in steps of 8 through
// double-buffered shared memory (the next step's elements are loaded into
// registers while the current step is multiplied).  Thread (tx, ty) owns rows
// {4ty..4ty+3, 64+4ty..64+4ty+3} and the same columns in tx: four 4 x 4 blocks,
// read from shared memory as float4 without bank conflicts.
constexpr int kGM = 128, kGN = 128, kGK = 8;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_kernel(GemmArgs a)
{
    __shared__ __align__(16) float As[2][kGK][kGM];
    __shared__ __align__(16) float Bs[2][kGK][kGN];
    const int bm = blockIdx.y * kGM, bn = blockIdx.x * kGN;
    const int kchunk = ((a.K + gridDim.z - 1) / gridDim.z + kGK - 1) / kGK * kGK;
    const int k0 = blockIdx.z * kchunk, k1 = min(a.K, k0 + kchunk);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float ra[4], rb[4];
    // element l of this thread's share of the (kk) step: A(m, k) and B(k, n)
    auto load = [&](int kk) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int idx = threadIdx.x + l * 256;
            int m, k, n, k2;
            if (!TA) { m = idx / kGK; k = idx % kGK; } else { k = idx / kGM; m = idx % kGM; }
            if (!TB) { k2 = idx / kGN; n = idx % kGN; } else { n = idx / kGK; k2 = idx % kGK; }
            const int gm = bm + m, gk = kk + k, gn = bn + n, gk2 = kk + k2;
            ra[l] = gm < a.M && gk < k1 ? (TA ? a.A[(size_t)gk * a.lda + gm] : a.A[(size_t)gm * a.lda + gk]) : 0.f;
            rb[l] = gn < a.N && gk2 < k1 ? (TB ? a.B[(size_t)gn * a.ldb + gk2] : a.B[(size_t)gk2 * a.ldb + gn]) : 0.f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int idx = threadIdx.x + l * 256;
            int m, k, n, k2;
            if (!TA) { m = idx / kGK; k = idx % kGK; } else { k = idx / kGM; m = idx % kGM; }
            if (!TB) { k2 = idx / kGN; n = idx % kGN; } else { n = idx / kGK; k2 = idx % kGK; }
            As[buf][k][m] = ra[l];
            Bs[buf][k2][n] = rb[l];
        }
    };
    float acc[8][8] = {};
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
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][4 * ty]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + 4 * ty]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][4 * tx]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + 4 * tx]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = bm + (i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4);
        if (m >= a.M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = bn + (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4);
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

// 64 x 64 output tile per block of 256 threads (4 x 4 per thread), K in steps
// of 16: the form for products with a side of 64 or less (the first layer, the
// input gradient, the first layer's weight gradient), where a 128-wide tile
// would compute mostly padding.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) sgemm_small_kernel(GemmArgs a)
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

template <bool TA, bool TB>
void sgemm_launch(const GemmArgs& a, int ksplit, cudaStream_t s)
{
    const int z = ksplit > 0 ? ksplit : 1;
    if (a.M > 64 && a.N > 64) {
        const dim3 grid((a.N + kGN - 1) / kGN, (a.M + kGM - 1) / kGM, z);
        sgemm_kernel<TA, TB><<<grid, 256, 0, s>>>(a);
    } else {
        const dim3 grid((a.N + 63) / 64, (a.M + 63) / 64, z);
        sgemm_small_kernel<TA, TB><<<grid, 256, 0, s>>>(a);
    }
}

// One launch: the 128 x 128 form when both output sides exceed 64, else the
// 64 x 64 form; ksplit > 1 splits K over gridDim.z (with a.atomic set).
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
