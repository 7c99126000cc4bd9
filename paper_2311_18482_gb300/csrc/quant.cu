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
    // gradient mode (quant_kernel<true>)
    const float* r;              // [N] utilisation ratio from the forward pass
    __nv_bfloat16* gtc;          // [N][kp] g_ij / |F_i^C|, code-major (feature index contiguous)
    __nv_bfloat16* gtd;          // [N][kp] g_ij / |F_i^D|
    long long kp;                // row stride of gtc / gtd (K rounded up to 8)
    float* u;                    // [2][N] sum_i g_ij cos^C_ij, sum_i g_ij cos^D_ij
    float cl, cc;                // lambda_lb / K, lambda_cos / K
};

struct Smem {
    unsigned char* a0;           // stage i's feature tile at a0 + i kATile
    unsigned char* b0;           // stage i's codebook tile at b0 + i bstride
    uint32_t bstride;
    uint64_t *full, *empty, *acc_full, *acc_empty, *norm_ready, *norm_free, *fin;
    float* norms;                // [2 slots][2][128] inverse feature norms
    float* xch;                  // [2 slots][2 halves][4][128] epilogue exchange
    float* rv;                   // [N] utilisation ratio (gradient mode)
    float* inv_s;                // [2][N]
    unsigned* cnt;               // [N]
    uint32_t* tmem_slot;
};

__host__ __device__ constexpr uint32_t quant_smem_bytes(int N)
{
    return 1024 + kStages * (kATile + (uint32_t)N * kChunk * 2) + 2 * 2 * kRows * 4 + 2 * 8 * kRows * 4 + N * 4 +
           2 * N * 4 + N * 4 + 8 +
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
    p += 2 * 8 * kRows * 4;
    s.rv = reinterpret_cast<float*>(p);
    p += N * 4;
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

template <bool GRAD>
__global__ void __launch_bounds__(kThreads, 1) quant_kernel(const __grid_constant__ CUtensorMap tmap_f,
                                                            const __grid_constant__ CUtensorMap tmap_s, QuantArgs q)
{
    extern __shared__ unsigned char smem_raw[];
    const int N = q.N;
    Smem s = carve(smem_raw, N);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) s.inv_s[i] = q.inv_s[i];
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        s.cnt[i] = 0u;
        if (GRAD) s.rv[i] = q.r[i];
    }
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
        float psum[4], usum[4];   // softmax column sums (gradient mode: sums of g cos^C, g cos^D)
#pragma unroll
        for (int i = 0; i < 4; ++i) psum[i] = usum[i] = 0.f;
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
            if constexpr (GRAD) {
                // pass 1: D, argmax, sum of exp(D) and of exp(D) r_j (for sigma_i = sum_k s_ik r_k)
                const float aC0 = s.norms[slot * 2 * kRows + r], aD0 = s.norms[slot * 2 * kRows + kRows + r];
                float best = -INFINITY, esum = 0.f, esr = 0.f;
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
                        const float e = __expf(dv);
                        esum += e;
                        esr = fmaf(e, s.rv[j0 + k], esr);
                    }
                }
                float* x = s.xch + slot * 8 * kRows;
                x[(4 * h) * kRows + r] = best;
                x[(4 * h + 1) * kRows + r] = __int_as_float(bi);
                x[(4 * h + 2) * kRows + r] = esum;
                x[(4 * h + 3) * kRows + r] = esr;
                named_sync(1 + quad, 64);
                const float ob = x[(4 * (1 - h)) * kRows + r];
                const int oi = __float_as_int(x[(4 * (1 - h) + 1) * kRows + r]);
                esum += x[(4 * (1 - h) + 2) * kRows + r];
                esr += x[(4 * (1 - h) + 3) * kRows + r];
                if (h == 0 ? ob > best : ob >= best) bi = oi;
                const float inv_e = valid ? 1.0f / esum : 0.f;
                const float sigma = esr * inv_e;
                // pass 2: g_ij = lambda_lb/K s_ij (r_j - sigma_i) - lambda_cos/K [j = m_i];
                // u^C_j += g cos^C_ij, u^D_j += g cos^D_ij; G^T scaled by the inverse feature norms
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const int c = c_lo + cc;
                    if (c >= c_hi) break;
                    const int j0 = 16 * c;
                    float vc[16], vd[16];
                    tmem_ld16(acc + j0, vc);
                    tmem_ld16(acc + N + j0, vd);
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const float cosc = vc[k] * aC0 * s.inv_s[j0 + k], cosd = vd[k] * aD0 * s.inv_s[N + j0 + k];
                        const float sv = __expf(fmaf(q.lambda_d, cosd, cosc)) * inv_e;
                        float g = q.cl * sv * (s.rv[j0 + k] - sigma);
                        if (j0 + k == bi) g -= q.cc;
                        g = valid ? g : 0.f;
                        if (valid) {
                            q.gtc[(size_t)(j0 + k) * q.kp + row] = __float2bfloat16_rn(g * aC0);
                            q.gtd[(size_t)(j0 + k) * q.kp + row] = __float2bfloat16_rn(g * aD0);
                        }
                        vc[k] = valid ? g * cosc : 0.f;     // rows past K: cos is NaN
                        vd[k] = valid ? g * cosd : 0.f;
                    }
                    psum[cc] += warp_colsum16(vc, lane);
                    usum[cc] += warp_colsum16(vd, lane);
                }
                fence_before();
                mbar_arrive(s.acc_empty + slot);
            } else {
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
        }
        // flush this warp's partial sums
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lcos += __shfl_xor_sync(0xffffffffu, lcos, o);
        if (ok) {
            if (GRAD) {
                if ((lane & 1) == 0)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc)
                        if (c_lo + cc < c_hi) {
                            atomicAdd(q.u + 16 * (c_lo + cc) + (lane >> 1), psum[cc]);
                            atomicAdd(q.u + N + 16 * (c_lo + cc) + (lane >> 1), usum[cc]);
                        }
            } else {
                if (lane == 0 && h == 0) atomicAdd(q.lcos, lcos);
                if ((lane & 1) == 0)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc)
                        if (c_lo + cc < c_hi) atomicAdd(q.psum + 16 * (c_lo + cc) + (lane >> 1), psum[cc]);
            }
        }
    }
    fence_before();
    const bool bad = __syncthreads_or(!ok);
    fence_after();
    if (bad) {
        if (threadIdx.x == 0) atomicExch(&g_quant_error, 1);
    } else if (!GRAD) {
        for (int i = threadIdx.x; i < N; i += blockDim.x)
            if (s.cnt[i]) atomicAdd(q.count + i, s.cnt[i]);
    }
    if (warp == 1) tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------
// Codebook gradient, contraction over the features (split-K):
//   raw[j][e] += sum_i GT[j][i] F[i][e]   (GT = gtc for CLIP dims e, gtd for DINO dims)
// CTA (x, y): the 128 dims [128 x, 128 x + 128) and the y-th slice of the
// 64-feature chunks.  A = GT tile [128 codes x 64 features] (K-major, TMA,
// 128-byte swizzle; codes past N read as zero); B = F tile [64 features x 128
// dims] as two 64-dim TMA boxes, read MN-major (dims contiguous).  Each MMA
// covers one 64-dim swizzle atom column (N = 64), so the operand spans one
// atom along N and only the stride between 8-feature groups (1024 bytes)
// matters; it is written into both offset fields.  The accumulator (128 lanes
// = codes x 128 columns = dims) is added into raw with atomics at the end.
constexpr int kGStages = 4;
constexpr int kGThreads = 192;
constexpr uint32_t kGATile = 128 * kChunk * 2;       // 16 KB
constexpr uint32_t kGBBox = kChunk * kChunk * 2;     // 8 KB: 64 features x 64 dims

__device__ __forceinline__ uint64_t desc_sw128_mn(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(1024 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

struct GemmArgs {
    int N, d, dclip_tiles;       // codebook size, dims, 128-dim tiles in the CLIP part
    int nch_total, nch_split;    // 64-feature chunks in all, per split
    float* raw;                  // [N][d]
};

__global__ void __launch_bounds__(kGThreads, 1) quant_grad_gemm_kernel(const __grid_constant__ CUtensorMap tmap_gtc,
                                                                       const __grid_constant__ CUtensorMap tmap_gtd,
                                                                       const __grid_constant__ CUtensorMap tmap_f,
                                                                       GemmArgs g)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* A0 = base;                                   // kGStages x 16 KB
    unsigned char* B0 = base + kGStages * kGATile;              // kGStages x 16 KB
    uint64_t* full = reinterpret_cast<uint64_t*>(B0 + kGStages * 2 * kGBBox);
    uint64_t* empty = full + kGStages;
    uint64_t* done = empty + kGStages;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int dt = blockIdx.x;
    const bool clip = dt < g.dclip_tiles;
    const CUtensorMap* tmap_a = clip ? &tmap_gtc : &tmap_gtd;
    const int c0 = blockIdx.y * g.nch_split;
    const int c1 = min(g.nch_total, c0 + g.nch_split);
    const int nck = max(0, c1 - c0);
    if (threadIdx.x == 0) {
        for (int i = 0; i < kGStages; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tslot, 128);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(tslot);
    bool ok = true;
    if (warp == 0) {
        if (lane == 0) {
            int st = 0;
            uint32_t ph = 0;
            for (int c = 0; c < nck; ++c) {
                if (!wait_bar(empty + st, ph ^ 1)) {
                    ok = false;
                    break;
                }
                const int f0 = (c0 + c) * kChunk;
                mbar_expect_tx(full + st, kGATile + 2 * kGBBox);
                tma_load_2d(A0 + st * kGATile, tmap_a, f0, 0, full + st);
                tma_load_2d(B0 + st * 2 * kGBBox, &tmap_f, 128 * dt, f0, full + st);
                tma_load_2d(B0 + st * 2 * kGBBox + kGBBox, &tmap_f, 128 * dt + 64, f0, full + st);
                if (++st == kGStages) {
                    st = 0;
                    ph ^= 1;
                }
            }
            for (int i = 0; i < kGStages; ++i) {     // nothing may still be landing at exit
                int k = st - 1 - i;
                uint32_t kp = ph;
                if (k < 0) {
                    k += kGStages;
                    kp ^= 1;
                }
                (void)wait_bar(full + k, kp);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(64, false, true);
            int st = 0;
            uint32_t ph = 0;
            for (int c = 0; c < nck; ++c) {
                if (!wait_bar(full + st, ph)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint64_t da = desc_sw128(smem_u32(A0 + st * kGATile));
                const uint64_t db0 = desc_sw128_mn(smem_u32(B0 + st * 2 * kGBBox));
                const uint64_t db1 = desc_sw128_mn(smem_u32(B0 + st * 2 * kGBBox + kGBBox));
#pragma unroll
                for (int k = 0; k < kChunk / 16; ++k) {
                    const uint32_t accumulate = (c > 0 || k > 0) ? 1u : 0u;
                    // A: +32 bytes per 16 features (K-major swizzle row); B: +2 x 1024 bytes (two 8-feature groups)
                    mma(tmem, da + 2u * k, db0 + 128u * k, idesc, accumulate);
                    mma(tmem + 64, da + 2u * k, db1 + 128u * k, idesc, accumulate);
                }
                commit(empty + st);
                if (++st == kGStages) {
                    st = 0;
                    ph ^= 1;
                }
            }
            commit(done);
        }
    }
    // epilogue: warps 2-5 (TMEM lane quadrant warp % 4): codes 32 (warp % 4) + lane
    if (warp >= 2) {
        const bool got = wait_bar(done, 0);
        fence_after();
        const int j = 32 * (warp & 3) + lane;
        if (got && nck > 0) {
            for (int c0c = 0; c0c < 128; c0c += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + c0c, v);
                if (j < g.N)
#pragma unroll
                    for (int k = 0; k < 16; ++k) atomicAdd(g.raw + (size_t)j * g.d + 128 * dt + c0c + k, v[k]);
            }
        }
        ok = ok && got;
    } else if (warp == 1 && lane == 0) {
        ok = ok && wait_bar(done, 0);     // every MMA of ours has completed
    }
    fence_before();
    const bool bad = __syncthreads_or(!ok);
    fence_after();
    if (bad && threadIdx.x == 0) atomicExch(&g_quant_error, 1);
    if (warp == 1) tmem_dealloc(tmem, 128);
}

// dL/dS_j^C[e] = invS^C_j (raw[j][e] - u^C_j S_j[e] invS^C_j) for CLIP dims, and
// lambda_D invS^D_j (raw[j][e] - u^D_j S_j[e] invS^D_j) for DINO dims (S the BF16 codebook).
__global__ void quant_grad_finalize_kernel(const float* __restrict__ raw, const float* __restrict__ u,
                                           const __nv_bfloat16* __restrict__ Sb, const float* __restrict__ inv_s,
                                           int N, int d, int d_clip, float lambda_d, float* __restrict__ grad)
{
    const size_t n = (size_t)N * d;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i / d), e = (int)(i - (size_t)j * d);
        const bool cpart = e < d_clip;
        const float is = inv_s[(cpart ? 0 : N) + j];
        const float w = cpart ? 1.f : lambda_d;
        grad[i] = w * is * (raw[i] - u[(cpart ? 0 : N) + j] * __bfloat162float(Sb[i]) * is);
    }
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

// 2-D BF16 tensor [rows, cols] row-major (row stride `stride` elements, default
// cols; cols = 0 means cols = stride), box [box_rows, 64], 128-byte swizzle.
le_status make_map(CUtensorMap* map, const void* base, long long rows, int cols, int box_rows, long long stride = 0)
{
    EncodeTiled fn;
    le_status st = tensor_map_encoder(&fn);
    if (st != LE_OK) return st;
    if (stride == 0) stride = cols;
    if (cols == 0) cols = (int)stride;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)stride * 2};
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
    LE_TRACE("le_quantize_workspace");
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
    LE_TRACE("le_quantize");
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
    LE_CUDA(cudaFuncSetAttribute(quant_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = q.ntiles < sms ? q.ntiles : sms;
    quant_kernel<false><<<grid, kThreads, smem, s>>>(mf, ms, q);
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

namespace leg {
namespace {
struct QuantGradWs {
    QuantWs base;
    __nv_bfloat16 *gtc, *gtd;
    float *raw, *u;
    long long kp;
    size_t bytes;
};

QuantGradWs quant_grad_ws(void* p, long long K, int N, int d)
{
    QuantGradWs w;
    w.base = quant_ws(p, N, d);
    size_t off = w.base.bytes;
    auto take = [&](size_t b) {
        const size_t o = off;
        off += (b + 255) & ~size_t(255);
        return reinterpret_cast<unsigned char*>(p) + o;
    };
    w.kp = (K + 7) / 8 * 8;
    w.gtc = reinterpret_cast<__nv_bfloat16*>(take((size_t)N * w.kp * 2));
    w.gtd = reinterpret_cast<__nv_bfloat16*>(take((size_t)N * w.kp * 2));
    w.raw = reinterpret_cast<float*>(take((size_t)N * d * 4 + (size_t)2 * N * 4));
    w.u = w.raw + (size_t)N * d;
    w.bytes = off;
    return w;
}
}  // namespace
}  // namespace leg

extern "C" le_status le_quantize_grad_workspace(int64_t K, int32_t n_cb, int32_t d, size_t* bytes)
{
    LE_TRACE("le_quantize_grad_workspace");
    LE_CHECK_ARG(bytes != nullptr, "bytes is null");
    LE_CHECK_ARG(K >= 1 && n_cb > 0 && d > 0, "bad sizes");
    *bytes = quant_grad_ws(nullptr, K, n_cb, d).bytes;
    return LE_OK;
}

extern "C" le_status le_quantize_grad(int64_t K, int32_t d, int32_t d_clip, const uint16_t* features, int32_t n_cb,
                                      const float* codebook, const float* r, float lambda_d, float lambda_cos,
                                      float lambda_lb, float* grad_codebook, void* workspace, size_t workspace_bytes,
                                      void* stream)
{
    LE_TRACE("le_quantize_grad");
    le_status st = check_quant(K, d, d_clip, n_cb);
    if (st != LE_OK) return st;
    if (d % 128 != 0 || d_clip % 128 != 0)
        LE_FAIL(LE_ERR_UNSUPPORTED, "codebook gradient: d = %d and d_clip = %d must be multiples of 128", d, d_clip);
    LE_CHECK_ARG(features && codebook && r && grad_codebook && workspace, "null pointer");
    LE_CHECK_ARG(aligned16(features), "features must be 16-byte aligned");
    LE_CHECK_ARG((reinterpret_cast<uintptr_t>(workspace) & 255u) == 0, "workspace must be 256-byte aligned");
    const QuantGradWs w = quant_grad_ws(workspace, K, n_cb, d);
    LE_CHECK_ARG(workspace_bytes >= w.bytes, "workspace has %zu bytes, needs %zu", workspace_bytes, w.bytes);
    cudaStream_t s = as_stream(stream);
    int dev = 0, sms = 0;
    LE_CUDA(cudaGetDevice(&dev));
    LE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUtensorMap mf, ms, mf64, mgc, mgd;
    if ((st = make_map(&mf, features, K, d, kRows)) != LE_OK) return st;
    if ((st = make_map(&ms, w.base.sb, (long long)kCopies * n_cb, d, n_cb)) != LE_OK) return st;
    if ((st = make_map(&mf64, features, K, d, kChunk)) != LE_OK) return st;
    if ((st = make_map(&mgc, w.gtc, n_cb, (int)K, 128, w.kp)) != LE_OK) return st;   // columns past K read as 0
    if ((st = make_map(&mgd, w.gtd, n_cb, (int)K, 128, w.kp)) != LE_OK) return st;
    LE_CUDA(cudaMemsetAsync(w.raw, 0, (size_t)n_cb * d * 4 + (size_t)2 * n_cb * 4, s));
    codebook_prep_kernel<<<n_cb, 128, 0, s>>>(codebook, d, d_clip, w.base.sb, w.base.inv_s, n_cb);
    LE_LAUNCHED();
    QuantArgs q{};
    q.K = K;
    q.N = n_cb;
    q.nchunks = d / kChunk;
    q.nclip = d_clip / kChunk;
    q.ntiles = (int)((K + kRows - 1) / kRows);
    q.lambda_d = lambda_d;
    q.inv_s = w.base.inv_s;
    q.r = r;
    q.gtc = w.gtc;
    q.gtd = w.gtd;
    q.kp = w.kp;
    q.u = w.u;
    q.cl = lambda_lb / (float)K;
    q.cc = lambda_cos / (float)K;
    const uint32_t smem = quant_smem_bytes(n_cb);
    LE_CUDA(cudaFuncSetAttribute(quant_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = q.ntiles < sms ? q.ntiles : sms;
    quant_kernel<true><<<grid, kThreads, smem, s>>>(mf, ms, q);
    LE_LAUNCHED();
    GemmArgs ga;
    ga.N = n_cb;
    ga.d = d;
    ga.dclip_tiles = d_clip / 128;
    ga.nch_total = (int)((K + kChunk - 1) / kChunk);
    const int dtiles = d / 128;
    const int splits = max(1, min(ga.nch_total, sms / dtiles));
    ga.nch_split = (ga.nch_total + splits - 1) / splits;
    ga.raw = w.raw;
    const uint32_t gsmem = 1024 + kGStages * (kGATile + 2 * kGBBox) + (2 * kGStages + 2) * 8;
    LE_CUDA(cudaFuncSetAttribute(quant_grad_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem));
    quant_grad_gemm_kernel<<<dim3(dtiles, splits), kGThreads, gsmem, s>>>(mgc, mgd, mf64, ga);
    LE_LAUNCHED();
    quant_grad_finalize_kernel<<<n_cb, 256, 0, s>>>(w.raw, w.u, w.base.sb, w.base.inv_s, n_cb, d, d_clip, lambda_d,
                                                    grad_codebook);
    LE_LAUNCHED();
    return LE_OK;
}
