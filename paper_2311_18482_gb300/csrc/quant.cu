// Quantisation of language features (Sec. 3.3 and the supplementary "Load
// Balancing Loss"):
//   D(F_i, f_j) = cos(F_i^C, f_j^C) + lambda_D cos(F_i^D, f_j^D)      (eq:q_dist)
//   m_i = argmax_j D(F_i, f_j) (ties -> lowest j)                      (eq:quant)
//   L_cos = mean_i (1 - cos^C(F_i, f_m)) + lambda_D (1 - cos^D(F_i, f_m))
//         = mean_i (1 + lambda_D - D(F_i, f_{m_i}))                    (eq:q_loss_cos)
//   r = counts of m / K, p = mean_i softmax_j D(F_i, f_j), L_lb = r . p (eq:q_loss_lb)
//   L_q = lambda_cos L_cos + lambda_lb L_lb                            (eq:q_loss_cb)
//
// quant_kernel (persistent, one CTA per SM, 10 warps): tiles of 128 features.
//   warp 0     TMA producer: per 64-column chunk, the feature tile [128 x 64]
//              and the codebook tile [N x 64] (BF16, 128-byte swizzle) into a
//              kStages-deep ring;
//   warp 1     tcgen05.mma issuer: CLIP chunks accumulate F^C S^C^T into TMEM
//              columns [0, N) of the tile's accumulator, DINO chunks F^D S^D^T
//              into [N, 2N); two accumulators alternate between tiles;
//   warps 2-5  feature norms: read every stage back (one row per thread) and
//              sum the squares of the CLIP and DINO parts;
//   warps 6-13 epilogue, one row per thread (TMEM lane) and half of the
//              columns per warp: D from the two dot products and the four
//              inverse norms, argmax, exp(D) (parked in the CLIP columns of
//              TMEM) and its sum; the halves combine through shared memory;
//              then the softmax column sums (a shuffle transposition per 16
//              columns, kept in registers across tiles), L_cos and the argmax
//              counts.
// Every mbarrier wait is bounded; on a timeout the kernel records it in
// g_quant_error (reported by le_device_status), stops and frees its TMEM.
#include <cuda.h>

#include "tc_common.cuh"

namespace leg {

// Set when quant_kernel gives up on a bounded wait (this translation unit's own
// flag; le_device_status reads it through quant_take_timeout).
__device__ int g_quant_error;

namespace {
using namespace tc;

constexpr int kStages = 5;
constexpr int kRows = 128;           // features per tile (MMA M)
constexpr int kChunk = 64;           // BF16 columns per stage (one 128-byte swizzle span)
constexpr uint32_t kATile = kRows * kChunk * 2;
constexpr int kThreads = 448;
// Every CTA reads the whole BF16 codebook once per tile from L2.  To keep 152
// SMs from hammering the same L2 lines at the same moment, the prep kernel
// writes kCopies copies (CTA b reads copy b % kCopies) and each CTA walks the
// 64-column chunks of each part starting at its own offset.
constexpr int kCopies = 8;

// K-major operand in the 128-byte swizzled layout TMA writes: 8-row atoms of
// 1024 bytes (SBO), version 1, layout type 2 (SWIZZLE_128B).  A 16-column K
// step moves the start address by 32 bytes.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

struct QuantArgs {
    long long K;
    int N, nchunks, nclip;       // codebook size, 64-column chunks, of which CLIP
    int ntiles;
    float lambda_d;
    const float* inv_s;          // [2][N] inverse norms of the BF16 codebook (CLIP, DINO)
    int32_t* m_out;              // [K]
    float* psum;                 // [N] column sums of the softmax
    unsigned* count;             // [N] argmax counts
    float* lcos;                 // [1] sum of 1 + lambda_D - D_max
};

struct Smem {
    unsigned char* a0;           // stage i's feature tile at a0 + i kATile
    unsigned char* b0;           // stage i's codebook tile at b0 + i bstride
    uint32_t bstride;
    uint64_t *full, *empty, *acc_full, *acc_empty, *norm_ready, *norm_free, *fin;
    float* norms;                // [2 slots][2][128] inverse feature norms
    float* xch;                  // [2 slots][2 halves][3][128] epilogue exchange
    float* inv_s;                // [2][N]
    unsigned* cnt;               // [N]
    uint32_t* tmem_slot;
};

__host__ __device__ constexpr uint32_t quant_smem_bytes(int N)
{
    return 1024 + kStages * (kATile + (uint32_t)N * kChunk * 2) + 2 * 2 * kRows * 4 + 2 * 6 * kRows * 4 + 2 * N * 4 +
           N * 4 + 8 +
           (2 * kStages + 10) * 8;
}

__device__ Smem carve(unsigned char* base, int N)
{
    Smem s;
    unsigned char* p = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(base) + 1023) & ~uintptr_t(1023));
    s.a0 = p;
    p += kStages * kATile;
    s.b0 = p;
    s.bstride = (uint32_t)N * kChunk * 2;    // a multiple of 1024 for N % 8 == 0
    p += kStages * s.bstride;
    s.norms = reinterpret_cast<float*>(p);
    p += 2 * 2 * kRows * 4;
    s.xch = reinterpret_cast<float*>(p);
    p += 2 * 6 * kRows * 4;
    s.inv_s = reinterpret_cast<float*>(p);
    p += 2 * N * 4;
    s.cnt = reinterpret_cast<unsigned*>(p);
    p += N * 4;
    uint64_t* bar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(p) + 7) & ~uintptr_t(7));
    s.full = bar;
    s.empty = bar + kStages;
    s.acc_full = bar + 2 * kStages;
    s.acc_empty = s.acc_full + 2;
    s.norm_ready = s.acc_full + 4;
    s.norm_free = s.acc_full + 6;
    s.fin = bar + 2 * kStages + 8;
    s.tmem_slot = reinterpret_cast<uint32_t*>(bar + 2 * kStages + 9);
    return s;
}

// Bounded wait (about a second, as tc::mbar_wait) that lets the waiting
// thread sleep in the barrier until the phase completes instead of spinning,
// so waiting roles leave issue slots to the epilogue.
__device__ __forceinline__ bool wait_bar(uint64_t* m, uint32_t parity)
{
    const uint32_t a = smem_u32(m);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity), "r"(0x989680u)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1ll << 31)) return false;
    }
}

__device__ __forceinline__ void named_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// One stage of a 16-value recursive-halving sum across the warp (see render.cu).
template <int N, int O>
__device__ __forceinline__ void halve(float* v, bool upper)
{
    constexpr int H = N / 2;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float lo = v[i], hi = v[i + H];
        const float recv = __shfl_xor_sync(0xffffffffu, upper ? lo : hi, O);
        v[i] = (upper ? hi : lo) + recv;
    }
}

// Column sums over the warp's 32 rows of 16 values: afterwards lanes 2c and
// 2c + 1 both hold the sum of column c.
__device__ __forceinline__ float warp_colsum16(float* v, int lane)
{
    halve<16, 16>(v, lane & 16);
    halve<8, 8>(v, lane & 8);
    halve<4, 4>(v, lane & 4);
    halve<2, 2>(v, lane & 2);
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// The i-th chunk this CTA processes within a tile: the CLIP chunks [0, nclip)
// first, then the DINO chunks, each part rotated by the CTA's offset.
__device__ __forceinline__ int chunk_at(int i, int nclip, int nchunks, int rot)
{
    const int nd = nchunks - nclip;
    return i < nclip ? (i + rot) % nclip : nclip + (i - nclip + rot) % nd;
}

__global__ void __launch_bounds__(kThreads, 1) quant_kernel(const __grid_constant__ CUtensorMap tmap_f,
                                                            const __grid_constant__ CUtensorMap tmap_s, QuantArgs q)
{
    extern __shared__ unsigned char smem_raw[];
    const int N = q.N;
    Smem s = carve(smem_raw, N);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) s.inv_s[i] = q.inv_s[i];
    for (int i = threadIdx.x; i < N; i += blockDim.x) s.cnt[i] = 0u;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(s.full + i, 1);
            mbar_init(s.empty + i, 1 + kRows);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(s.acc_full + i, 1);
            mbar_init(s.acc_empty + i, 2 * kRows);
            mbar_init(s.norm_ready + i, kRows);
            mbar_init(s.norm_free + i, 2 * kRows);
        }
        mbar_init(s.fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t ncols = 32;
    while (ncols < 4u * N) ncols <<= 1;
    if (warp == 1) tmem_alloc(s.tmem_slot, ncols);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(s.tmem_slot);
    const uint32_t b_bytes = (uint32_t)N * kChunk * 2;
    bool ok = true;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int st = 0;
            uint32_t ph = 0;
            for (int t = blockIdx.x; t < q.ntiles && ok; t += gridDim.x) {
                for (int c = 0; c < q.nchunks; ++c) {
                    if (!wait_bar(s.empty + st, ph ^ 1)) {
                        ok = false;
                        break;
                    }
                    const int cc = chunk_at(c, q.nclip, q.nchunks, blockIdx.x);
                    mbar_expect_tx(s.full + st, kATile + b_bytes);
                    tma_load_2d(s.a0 + st * kATile, &tmap_f, cc * kChunk, t * kRows, s.full + st);
                    tma_load_2d(s.b0 + st * s.bstride, &tmap_s, cc * kChunk, (blockIdx.x % kCopies) * N, s.full + st);
                    if (++st == kStages) {
                        st = 0;
                        ph ^= 1;
                    }
                }
            }
            // nothing of ours may still be landing when the CTA exits (on the normal
            // path every fill has been consumed and these waits return at once)
            for (int i = 0; i < kStages; ++i) {
                int k = st - 1 - i;
                uint32_t kp = ph;
                if (k < 0) {
                    k += kStages;
                    kp ^= 1;
                }
                (void)wait_bar(s.full + k, kp);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(N, false, false);
            int st = 0;
            uint32_t ph = 0;
            int it = 0;
            for (int t = blockIdx.x; t < q.ntiles && ok; t += gridDim.x, ++it) {
                const int slot = it & 1;
                const uint32_t aph = (uint32_t)(it >> 1) & 1u;
                if (!wait_bar(s.acc_empty + slot, aph ^ 1)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t acc = tmem + (uint32_t)(2 * N * slot);
                for (int c = 0; c < q.nchunks; ++c) {
                    if (!wait_bar(s.full + st, ph)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const bool clip = c < q.nclip;
                    const uint32_t d = acc + (clip ? 0u : (uint32_t)N);
                    const uint64_t da = desc_sw128(smem_u32(s.a0 + st * kATile)),
                                   db = desc_sw128(smem_u32(s.b0 + st * s.bstride));
#pragma unroll
                    for (int k = 0; k < kChunk / 16; ++k) {
                        const uint32_t accumulate = (k > 0 || (c != 0 && c != q.nclip)) ? 1u : 0u;
                        mma(d, da + 2u * k, db + 2u * k, idesc, accumulate);
                    }
                    commit(s.empty + st);
                    if (++st == kStages) {
                        st = 0;
                        ph ^= 1;
                    }
                }
                if (!ok) break;
                commit(s.acc_full + slot);
            }
            commit(s.fin);
            (void)wait_bar(s.fin, 0);      // every MMA of ours has completed
        }
    } else if (warp < 6) {
        // ---------------- feature norms: row r = 32 (warp - 2) + lane
        const int r = 32 * (warp - 2) + lane;
        int st = 0;
        uint32_t ph = 0;
        int it = 0;
        for (int t = blockIdx.x; t < q.ntiles && ok; t += gridDim.x, ++it) {
            float sc = 0.f, sd = 0.f;
            for (int c = 0; c < q.nchunks; ++c) {
                if (!wait_bar(s.full + st, ph)) {
                    ok = false;
                    break;
                }
                // row r of the swizzled tile: 16-byte chunk j sits at (j ^ (r & 7)); reading
                // chunk (i + r) & 7 at step i keeps eight consecutive rows on distinct banks
                const unsigned char* row = s.a0 + st * kATile + r * 128;
                float acc = 0.f;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const uint4 u = *reinterpret_cast<const uint4*>(row + (((i + r) & 7) << 4));
                    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float2 f = __bfloat1622float2(h[k]);
                        acc = fmaf(f.x, f.x, fmaf(f.y, f.y, acc));
                    }
                }
                if (c < q.nclip)
                    sc += acc;
                else
                    sd += acc;
                mbar_arrive(s.empty + st);
                if (++st == kStages) {
                    st = 0;
                    ph ^= 1;
                }
            }
            if (!ok) break;
            const int slot = it & 1;
            if (!wait_bar(s.norm_free + slot, ((uint32_t)(it >> 1) & 1u) ^ 1u)) {
                ok = false;
                break;
            }
            s.norms[slot * 2 * kRows + r] = 1.0f / sqrtf(sc);
            s.norms[slot * 2 * kRows + kRows + r] = 1.0f / sqrtf(sd);
            mbar_arrive(s.norm_ready + slot);
        }
    } else {
        // ---------------- epilogue: row = TMEM lane 32 (warp % 4) + lane; half h of the
        // 16-column chunks (h = 0: chunks [0, nh0), h = 1: [nh0, N/16))
        const int quad = warp & 3, h = (warp - 6) >> 2;
        const int r = 32 * quad + lane;
        const uint32_t lanef = (uint32_t)(32 * quad) << 16;
        const int nch = N / 16, nh0 = (nch + 1) / 2;
        const int c_lo = h ? nh0 : 0, c_hi = h ? nch : nh0;
        float psum[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) psum[i] = 0.f;
        float lcos = 0.f;
        int it = 0;
        for (int t = blockIdx.x; t < q.ntiles && ok; t += gridDim.x, ++it) {
            const int slot = it & 1;
            const uint32_t aph = (uint32_t)(it >> 1) & 1u;
            // the two warps of a quadrant decide together, so that a timeout never
            // leaves one of them at the exchange barrier below
            const bool got = wait_bar(s.norm_ready + slot, aph) && wait_bar(s.acc_full + slot, aph);
            if (bar_any(1 + quad, 64, !got)) {
                ok = false;
                break;
            }
            fence_after();
            const float aC = s.norms[slot * 2 * kRows + r];
            const float aD = q.lambda_d * s.norms[slot * 2 * kRows + kRows + r];
            mbar_arrive(s.norm_free + slot);
            const long long row = (long long)t * kRows + r;
            const bool valid = row < q.K;
            const uint32_t acc = tmem + lanef + (uint32_t)(2 * N * slot);
            // pass 1 over this half's columns: D, argmax (first maximum), sum of
            // exp(D) (|D| <= 1 + lambda_D: no shift needed); exp(D) replaces the
            // CLIP dot products in TMEM for pass 2
            float best = -INFINITY, esum = 0.f;
            int bi = 0;
            for (int c = c_lo; c < c_hi; ++c) {
                const int j0 = 16 * c;
                float vc[16], vd[16];
                tmem_ld16(acc + j0, vc);
                tmem_ld16(acc + N + j0, vd);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const float dv = fmaf(vc[k] * aC, s.inv_s[j0 + k], vd[k] * aD * s.inv_s[N + j0 + k]);
                    if (dv > best) {
                        best = dv;
                        bi = j0 + k;
                    }
                    vc[k] = __expf(dv);
                    esum += vc[k];
                }
                tmem_st16(acc + j0, vc);
            }
            // combine the halves (ties -> half 0, the lower indices)
            float* x = s.xch + slot * 6 * kRows;
            x[(3 * h) * kRows + r] = best;
            x[(3 * h + 1) * kRows + r] = __int_as_float(bi);
            x[(3 * h + 2) * kRows + r] = esum;
            named_sync(1 + quad, 64);
            const float ob = x[(3 * (1 - h)) * kRows + r];
            const int oi = __float_as_int(x[(3 * (1 - h) + 1) * kRows + r]);
            esum += x[(3 * (1 - h) + 2) * kRows + r];
            if (h == 0 ? ob > best : ob >= best) {
                best = ob;
                bi = oi;
            }
            const float inv_e = valid ? 1.0f / esum : 0.f;
            tmem_wait_st();
            // pass 2: softmax column sums of this half's columns over the warp's 32 rows
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int c = c_lo + cc;
                if (c >= c_hi) break;
                float e[16];
                tmem_ld16(acc + 16 * c, e);
#pragma unroll
                for (int k = 0; k < 16; ++k) e[k] = valid ? e[k] * inv_e : 0.f;   // rows past K hold NaN
                psum[cc] += warp_colsum16(e, lane);
            }
            fence_before();
            mbar_arrive(s.acc_empty + slot);
            if (valid && h == 0) {
                q.m_out[row] = bi;
                lcos += 1.0f + q.lambda_d - best;
                atomicAdd(s.cnt + bi, 1u);
            }
        }
        // flush this warp's partial sums
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lcos += __shfl_xor_sync(0xffffffffu, lcos, o);
        if (ok) {
            if (lane == 0 && h == 0) atomicAdd(q.lcos, lcos);
            if ((lane & 1) == 0)
#pragma unroll
                for (int cc = 0; cc < 4; ++cc)
                    if (c_lo + cc < c_hi) atomicAdd(q.psum + 16 * (c_lo + cc) + (lane >> 1), psum[cc]);
        }
    }
    fence_before();
    const bool bad = __syncthreads_or(!ok);
    fence_after();
    if (bad) {
        if (threadIdx.x == 0) atomicExch(&g_quant_error, 1);
    } else {
        for (int i = threadIdx.x; i < N; i += blockDim.x)
            if (s.cnt[i]) atomicAdd(q.count + i, s.cnt[i]);
    }
    if (warp == 1) tmem_dealloc(tmem, ncols);
}

// BF16 copies of the codebook (round to nearest even; kCopies stacked copies)
// and the inverse norms of its CLIP and DINO parts, computed from the rounded
// values.  One block per code.
__global__ void codebook_prep_kernel(const float* __restrict__ S, int d, int d_clip, __nv_bfloat16* __restrict__ Sb,
                                     float* __restrict__ inv_s, int N)
{
    const int j = blockIdx.x;
    float sc = 0.f, sd = 0.f;
    for (int e = threadIdx.x; e < d; e += blockDim.x) {
        const __nv_bfloat16 h = __float2bfloat16_rn(S[(size_t)j * d + e]);
#pragma unroll
        for (int c = 0; c < kCopies; ++c) Sb[((size_t)c * N + j) * d + e] = h;
        const float v = __bfloat162float(h);
        if (e < d_clip)
            sc = fmaf(v, v, sc);
        else
            sd = fmaf(v, v, sd);
    }
    __shared__ float red[2][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sc += __shfl_xor_sync(0xffffffffu, sc, o);
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sc;
        red[1][threadIdx.x >> 5] = sd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f, b = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += red[0][w];
            b += red[1][w];
        }
        inv_s[j] = 1.0f / sqrtf(a);
        inv_s[N + j] = 1.0f / sqrtf(b);
    }
}

// r = counts / K, p = psum / K, L_lb = r . p, L_cos = lcos / K, L_q.
__global__ void quant_finalize_kernel(const float* __restrict__ psum, const unsigned* __restrict__ count,
                                      const float* __restrict__ lcos, int N, long long K, float lambda_cos,
                                      float lambda_lb, float* __restrict__ r_out, float* __restrict__ p_out,
                                      float* __restrict__ loss)
{
    __shared__ float red[32];
    const float invK = 1.0f / (float)K;
    float lb = 0.f;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const float r = (float)count[j] * invK, p = psum[j] * invK;
        if (r_out) r_out[j] = r;
        if (p_out) p_out[j] = p;
        lb = fmaf(r, p, lb);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lb += __shfl_xor_sync(0xffffffffu, lb, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lb;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        const float lc = lcos[0] * invK;
        loss[0] = lambda_cos * lc + lambda_lb * t;
        loss[1] = lc;
        loss[2] = t;
    }
}

#define LE_FAIL(status, ...)          \
    do {                              \
        ::leg::set_error(__VA_ARGS__); \
        return status;                \
    } while (0)

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

le_status encoder(EncodeTiled* fn)
{
    static EncodeTiled cached = nullptr;
    if (!cached) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) !=
                cudaSuccess ||
            qr != cudaDriverEntryPointSuccess || !p)
            LE_FAIL(LE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
        cached = reinterpret_cast<EncodeTiled>(p);
    }
    *fn = cached;
    return LE_OK;
}

// 2-D BF16 tensor [rows, cols] row-major, box [box_rows, 64], 128-byte swizzle.
le_status make_map(CUtensorMap* map, const void* base, long long rows, int cols, int box_rows)
{
    EncodeTiled fn;
    le_status st = encoder(&fn);
    if (st != LE_OK) return st;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kChunk, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) LE_FAIL(LE_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return LE_OK;
}

struct QuantWs {
    __nv_bfloat16* sb;
    float *inv_s, *psum, *lcos;
    unsigned* count;
    size_t bytes;
};

QuantWs quant_ws(void* base, int N, int d)
{
    QuantWs w;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off += (b + 255) & ~size_t(255);
        return reinterpret_cast<unsigned char*>(base) + o;
    };
    w.sb = reinterpret_cast<__nv_bfloat16*>(take((size_t)kCopies * N * d * 2));
    w.inv_s = reinterpret_cast<float*>(take((size_t)2 * N * 4));
    w.psum = reinterpret_cast<float*>(take((size_t)N * 4 + (size_t)N * 4 + 4));
    w.count = reinterpret_cast<unsigned*>(w.psum + N);
    w.lcos = reinterpret_cast<float*>(w.count + N);
    w.bytes = off;
    return w;
}

le_status check_quant(long long K, int d, int d_clip, int N)
{
    LE_CHECK_ARG(K >= 1, "K = %lld < 1", K);
    LE_CHECK_ARG(K < (1ll << 31), "K = %lld: at most 2^31 - 1 features per call", K);
    LE_CHECK_ARG(d > 0 && d_clip > 0 && d_clip < d, "need 0 < d_clip < d (d = %d, d_clip = %d)", d, d_clip);
    if (d % kChunk != 0 || d_clip % kChunk != 0)
        LE_FAIL(LE_ERR_UNSUPPORTED, "d = %d and d_clip = %d must be multiples of 64", d, d_clip);
    if (N < 16 || N > 128 || N % 16 != 0)
        LE_FAIL(LE_ERR_UNSUPPORTED, "n_cb = %d: supported codebook sizes are 16..128, multiples of 16", N);
    return LE_OK;
}

}  // namespace
}  // namespace leg

using namespace leg;

extern "C" le_status le_quantize_workspace(int32_t n_cb, int32_t d, size_t* bytes)
{
    LE_CHECK_ARG(bytes != nullptr, "bytes is null");
    LE_CHECK_ARG(n_cb > 0 && d > 0, "bad sizes");
    *bytes = quant_ws(nullptr, n_cb, d).bytes;
    return LE_OK;
}

extern "C" le_status le_quantize(int64_t K, int32_t d, int32_t d_clip, const uint16_t* features, int32_t n_cb,
                                 const float* codebook, float lambda_d, float lambda_cos, float lambda_lb,
                                 int32_t* indices, float* r, float* p, float* loss, void* workspace,
                                 size_t workspace_bytes, void* stream)
{
    le_status st = check_quant(K, d, d_clip, n_cb);
    if (st != LE_OK) return st;
    LE_CHECK_ARG(features && codebook && indices && loss && workspace, "null pointer");
    LE_CHECK_ARG(aligned16(features), "features must be 16-byte aligned");
    LE_CHECK_ARG((reinterpret_cast<uintptr_t>(workspace) & 255u) == 0, "workspace must be 256-byte aligned");
    const QuantWs w = quant_ws(workspace, n_cb, d);
    LE_CHECK_ARG(workspace_bytes >= w.bytes, "workspace has %zu bytes, needs %zu", workspace_bytes, w.bytes);
    cudaStream_t s = as_stream(stream);
    int dev = 0, sms = 0;
    LE_CUDA(cudaGetDevice(&dev));
    LE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUtensorMap mf, ms;
    if ((st = make_map(&mf, features, K, d, kRows)) != LE_OK) return st;
    if ((st = make_map(&ms, w.sb, (long long)kCopies * n_cb, d, n_cb)) != LE_OK) return st;
    LE_CUDA(cudaMemsetAsync(w.psum, 0, (size_t)n_cb * 8 + 4, s));
    codebook_prep_kernel<<<n_cb, 128, 0, s>>>(codebook, d, d_clip, w.sb, w.inv_s, n_cb);
    LE_LAUNCHED();
    QuantArgs q;
    q.K = K;
    q.N = n_cb;
    q.nchunks = d / kChunk;
    q.nclip = d_clip / kChunk;
    q.ntiles = (int)((K + kRows - 1) / kRows);
    q.lambda_d = lambda_d;
    q.inv_s = w.inv_s;
    q.m_out = indices;
    q.psum = w.psum;
    q.count = w.count;
    q.lcos = w.lcos;
    const uint32_t smem = quant_smem_bytes(n_cb);
    LE_CUDA(cudaFuncSetAttribute(quant_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = q.ntiles < sms ? q.ntiles : sms;
    quant_kernel<<<grid, kThreads, smem, s>>>(mf, ms, q);
    LE_LAUNCHED();
    quant_finalize_kernel<<<1, 128, 0, s>>>(w.psum, w.count, w.lcos, n_cb, K, lambda_cos, lambda_lb, r, p, loss);
    LE_LAUNCHED();
    return LE_OK;
}

namespace leg {
// Reads and clears the quantisation kernel's timeout record.
le_status quant_take_timeout(bool* timed_out)
{
    int flag = 0;
    LE_CUDA(cudaMemcpyFromSymbol(&flag, g_quant_error, sizeof(int)));
    if (flag) {
        const int zero = 0;
        LE_CUDA(cudaMemcpyToSymbol(g_quant_error, &zero, sizeof(int)));
    }
    *timed_out = flag != 0;
    return LE_OK;
}
}  // namespace leg
