// The decoder network at the widths of supp. Tab. dmlp -- 8 -> 128 -> 256 -> N,
// ReLU after the first two layers (Eq. eq:lem_dec; D_MLP is a stack of 1x1
// convolutions, i.e. a per-pixel MLP) -- on the tensor cores (tcgen05, BF16
// operands, FP32 accumulation in TMEM).
//
// At these widths the weights alone take 132 KB of BF16 (196 KB for 256
// codes), so the two-tiles-in-flight plan of decoder_tc.cu does not fit.  One
// persistent CTA per SM, one tile in flight, four warpgroups: thread t serves
// row t % 128 of the 128-pixel tile (TMEM lane) and the columns of part t / 128
// in every epilogue; thread 0 also issues the MMAs and bulk copies:
//   weights      BF16 canonical images of W1 [128 x 16] (input padded to 16),
//                W2 [256 x 128] and W3 [N x 256], prepared once per call in the
//                caller's workspace and copied into shared memory once per CTA;
//                for 128 < N <= 256 (inference only) W3's two 128-code halves
//                take turns in one 64 KB slot, in alternating order from tile
//                to tile so that one half is copied per tile.
//   activations  one 64 KB region holds the operand of the next MMA stage --
//                H1, H2 and, training, dZ, dH2, dH1 -- each written by the
//                epilogue once the MMAs reading its predecessor have completed;
//                the ReLU masks of h1 and h2 are kept as bits (4 + 8 words per
//                row, in shared memory so that the epilogue loops stay rolled).
//   TMEM         512 columns: [0, 256) hidden-layer accumulators (h1, h2, dh2,
//                dh1), [256, 256 + N) the logits, later [256, 272) dx.
// Training (N <= 128) takes two passes:
//   pass 1  wide_kernel<true>: forward, the uncertainty-weighted cross-entropy
//           (Eqs. eq:lem_loss_ce1, eq:lem_loss_uncer; dL/dz = dz / P with dz =
//           lambda_CE (1 - u) (softmax - onehot), dL/du = (lambda_u - lambda_CE
//           CE) / P) and the input-gradient chain dZ -> dH2 -> dH1 -> dX on the
//           tensor cores (the 1 / P is applied to dX and to the weight
//           gradients);
//           each operand image (X, H1, H2, dZ, dH2, dH1) leaves shared memory
//           by a bulk copy into the caller's workspace, one blob per tile;
//   pass 2  wide_wgrad_kernel: the weight and bias gradients, contractions
//           over the pixels of those images, split over CTAs by pixel tiles and
//           by output (dW3 | dW2 | dW1), accumulated in TMEM and added to the
//           outputs with atomics once per CTA.  Bias gradients are MMAs against
//           a ones operand (b3, b2) or the ones column 8 of X (b1).
// Every mbarrier wait is bounded (about a second); on timeout the kernel
// records it in g_wide_error (reported by le_device_status), stops and frees
// its TMEM.
#include "tc_common.cuh"

namespace leg {

__device__ int g_wide_error;

namespace {
using namespace tc;

constexpr int kW1 = 128, kW2 = 256;          // hidden widths (supp. Tab. dmlp)
constexpr int kRows = 128;                   // pixels per tile (MMA M)
constexpr uint32_t kW1Bytes = sbuf_bytes(kW1, 16), kW2Bytes = sbuf_bytes(kW2, kW1),
                   kW3Half = sbuf_bytes(128, kW2), kXBytes = sbuf_bytes(kRows, 16),
                   kABytes = sbuf_bytes(kRows, kW2);

// Shared memory of wide_kernel (offsets from a 1024-byte aligned base).
constexpr uint32_t kSW1 = 0, kSW2 = kSW1 + kW1Bytes, kSW3 = kSW2 + kW2Bytes, kSX = kSW3 + kW3Half,
                   kSA = kSX + kXBytes, kSBias = kSA + kABytes, kSMask = kSBias + (kW1 + kW2 + 256) * 4,
                   kSXch = kSMask + kRows * 12 * 4, kSBar = kSXch + 4 * kRows * 16, kSSlot = kSBar + 4 * 8,
                   kSmem = kSSlot + 16;

// One tile's operand images in the training workspace (pass 1 writes, pass 2 reads).
constexpr uint32_t kBX = 0, kBH1 = kBX + kXBytes, kBH2 = kBH1 + sbuf_bytes(kRows, kW1),
                   kBZ = kBH2 + sbuf_bytes(kRows, kW2), kBD2 = kBZ + sbuf_bytes(kRows, 128),
                   kBD1 = kBD2 + sbuf_bytes(kRows, kW2), kBlob = kBD1 + sbuf_bytes(kRows, kW1);

// TMEM column bases.
constexpr uint32_t kTH = 0, kTZ = 256;

struct WideArgs {
    int P, ncb;
    const float *feat, *unc;
    const int32_t* target;
    const float *b1, *b2, *b3;
    const unsigned char* img;        // W1 | W2 | W3 images
    float lambda_ce, lambda_u, invP;
    float* loss;
    float *d_feat, *d_unc;
    int32_t* argmax;
    float* prob;
    unsigned char* blobs;            // training: ntiles x kBlob
};

__device__ __forceinline__ void cta_publish()
{
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
}

// Four warpgroups serve the tile: thread t handles row t % 128 (TMEM lane) and
// the columns of part t / 128 in every epilogue.
constexpr int kParts = 4, kThreads = kParts * kRows;

// Wait for the MMA barrier (every thread); false for every thread if any timed out.
__device__ __forceinline__ bool wide_wait(uint64_t* bar, uint32_t& phase)
{
    const bool ok = mbar_wait(bar, phase);
    phase ^= 1u;
    const bool bad = bar_any(0, kThreads, !ok);
    if (bad && threadIdx.x == 0) atomicExch(&g_wide_error, 1);
    fence_after();
    return !bad;
}

// Accumulator columns [c0, c1) of this thread's row + bias, ReLU, stored as
// BF16 into the canonical buffer (C columns); bit j of the 16-bit mask half
// mask[c / 16] is set where column c + j is positive (mask: the row's halves
// in shared memory).
template <int C>
__device__ __forceinline__ void relu_epilogue(uint32_t tl, const float* bias, unsigned char* dst, int row, int c0,
                                              int c1, uint16_t* mask)
{
    float v[16];
#pragma unroll 1
    for (int c = c0; c < c1; c += 16) {
        tmem_ld16(tl + c, v);
        uint32_t bits = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            v[j] = fmaxf(v[j] + bias[c + j], 0.f);
            bits |= (v[j] > 0.f ? 1u : 0u) << j;
        }
        mask[c / 16] = (uint16_t)bits;
        sts_bf16x8(smem_u32(dst) + sbuf_off(row, c, C), v);
        sts_bf16x8(smem_u32(dst) + sbuf_off(row, c + 8, C), v + 8);
    }
}

// Accumulator columns [c0, c1) times the ReLU mask, stored as BF16 (the
// backward through a ReLU layer).
template <int C>
__device__ __forceinline__ void mask_epilogue(uint32_t tl, const uint16_t* mask, unsigned char* dst, int row, int c0,
                                              int c1)
{
    float v[16];
#pragma unroll 1
    for (int c = c0; c < c1; c += 16) {
        tmem_ld16(tl + c, v);
        const uint32_t bits = mask[c / 16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = ((bits >> j) & 1u) ? v[j] : 0.f;
        sts_bf16x8(smem_u32(dst) + sbuf_off(row, c, C), v);
        sts_bf16x8(smem_u32(dst) + sbuf_off(row, c + 8, C), v + 8);
    }
}

// Running maximum (first index on ties), sum of exp(z - max) and the target's
// logit over the logits (+ b3) of columns [c0, min(c1, ncb)).
__device__ __forceinline__ float4 part_lse(uint32_t tz, const float* b3, int c0, int c1, int ncb, int t)
{
    float m = -INFINITY, s = 0.f, zt = 0.f, v[16];
    int am = 0;
#pragma unroll 1
    for (int c = c0; c < c1 && c < ncb; c += 16) {
        tmem_ld16(tz + c, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float z = v[j] + b3[c + j];
            if (c + j == t) zt = z;
            if (z > m) {
                s = s * __expf(m - z) + 1.f;
                m = z;
                am = c + j;
            } else {
                s += __expf(z - m);
            }
        }
    }
    return make_float4(m, s, __int_as_float(am), zt);
}

template <bool TRAIN>
__global__ void __launch_bounds__(kThreads, 1) wide_kernel(WideArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* const sW1 = sm + kSW1;
    unsigned char* const sW2 = sm + kSW2;
    unsigned char* const sW3 = sm + kSW3;
    unsigned char* const sX = sm + kSX;
    unsigned char* const sA = sm + kSA;
    float* const bias = reinterpret_cast<float*>(sm + kSBias);
    const float *b1s = bias, *b2s = bias + kW1, *b3s = bias + kW1 + kW2;
    float4* const xch = reinterpret_cast<float4*>(sm + kSXch);          // [kParts][kRows]
    uint64_t* const bars = reinterpret_cast<uint64_t*>(sm + kSBar);   // 0 MMA done, 1 weights, 2 W3 half
    uint32_t* const slot = reinterpret_cast<uint32_t*>(sm + kSSlot);
    const int tid = threadIdx.x, row = tid & (kRows - 1), part = tid / kRows;
    uint16_t* const m1 = reinterpret_cast<uint16_t*>(sm + kSMask) + row * 24;   // h1: 8 halves
    uint16_t* const m2 = m1 + 8;                                                // h2: 16 halves
    const int ncb = a.ncb;
    const bool halves = ncb > 128;
    const uint32_t w3bytes = halves ? kW3Half : (uint32_t)ncb * kW2 * 2;
    const unsigned char* w3img = a.img + kW1Bytes + kW2Bytes;
    // this part's columns: 32 of h1, 64 of h2, a quarter of the logits (32 up to 128 codes, 64 beyond)
    const int h1c0 = part * (kW1 / kParts), h1c1 = h1c0 + kW1 / kParts;
    const int h2c0 = part * (kW2 / kParts), h2c1 = h2c0 + kW2 / kParts;
    const int zw = halves ? 64 : 32, zc0 = part * zw, zc1 = zc0 + zw;

    for (int i = tid; i < kW1 + kW2 + ncb; i += kThreads)
        bias[i] = i < kW1 ? a.b1[i] : (i < kW1 + kW2 ? a.b2[i - kW1] : a.b3[i - kW1 - kW2]);
    if (tid == 0) {
        for (int k = 0; k < 3; ++k) mbar_init(bars + k, 1);
        fence_proxy_async();
        mbar_expect_tx(bars + 1, kW1Bytes + kW2Bytes + w3bytes);
        bulk_g2s(sW1, a.img, kW1Bytes, bars + 1);
        bulk_g2s(sW2, a.img + kW1Bytes, kW2Bytes, bars + 1);
        bulk_g2s(sW3, w3img, w3bytes, bars + 1);
    }
    if (tid < 32) tmem_alloc(slot, 512);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(slot);
    const uint32_t tl = tbase + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16);   // this warp's TMEM lanes
    uint32_t ph = 0, ph3 = 0;
    int resident = 0;                     // the W3 half in the slot (halves only; thread 0)
    bool ok = mbar_wait(bars + 1, 0);
    if (bar_any(0, kThreads, !ok)) {
        if (tid == 0) atomicExch(&g_wide_error, 1);
        ok = false;
    }
    float lce = 0.f, lu = 0.f;
    const int ntiles = (a.P + kRows - 1) / kRows;
    for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
        const int p = tile * kRows + row;
        const bool valid = p < a.P;
        unsigned char* blob = TRAIN ? a.blobs + (size_t)tile * kBlob : nullptr;
        // E0: X = [x | 1 | 0] (column 8 is the bias input of dW1's contraction)
        if (part == 0) {
            float x[16];
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = valid ? a.feat[(size_t)c * a.P + p] : 0.f;
#pragma unroll
            for (int c = 8; c < 16; ++c) x[c] = c == 8 ? 1.f : 0.f;
            sbuf_store8(SBuf{sX, 16}, row, 0, x);
            sbuf_store8(SBuf{sX, 16}, row, 8, x + 8);
        }
        cta_publish();
        if (tid == 0) {
            mma(tbase + kTH, kdesc_at(smem_u32(sX), 16, 0, 0), kdesc_at(smem_u32(sW1), 16, 0, 0),
                idesc_bf16(kW1, false, false), 0);
            commit(bars);
            if (TRAIN) {
                bulk_s2g(blob + kBX, sX, kXBytes);
                bulk_commit();
            }
        }
        if (!(ok = wide_wait(bars, ph))) break;
        // E1: H1 = relu(h1 + b1)
        relu_epilogue<kW1>(tl + kTH, b1s, sA, row, h1c0, h1c1, m1);
        cta_publish();
        if (tid == 0) {
            const uint32_t a0 = smem_u32(sA), w2 = smem_u32(sW2);
#pragma unroll
            for (int k = 0; k < kW1 / 16; ++k)
                mma(tbase + kTH, kdesc_at(a0, kW1, 0, 16 * k), kdesc_at(w2, kW1, 0, 16 * k),
                    idesc_bf16(kW2, false, false), k > 0);
            commit(bars);
            if (TRAIN) {
                bulk_s2g(blob + kBH1, sA, sbuf_bytes(kRows, kW1));
                bulk_commit();
                bulk_wait_read_all();       // H1's region is rewritten by E2
            }
        }
        if (!(ok = wide_wait(bars, ph))) break;
        // E2: H2 = relu(h2 + b2), over H1 (whose MMAs have completed)
        relu_epilogue<kW2>(tl + kTH, b2s, sA, row, h2c0, h2c1, m2);
        cta_publish();
        if (tid == 0) {
            const uint32_t a0 = smem_u32(sA), w3 = smem_u32(sW3);
            if (!halves) {
                const uint32_t id = idesc_bf16(ncb, false, false);
#pragma unroll 4
                for (int k = 0; k < kW2 / 16; ++k)
                    mma(tbase + kTZ, kdesc_at(a0, kW2, 0, 16 * k), kdesc_at(w3, kW2, 0, 16 * k), id, k > 0);
            } else {
                // the resident half first, then the other one copied into the slot
                for (int h = 0; h < 2; ++h) {
                    const int half = h == 0 ? resident : 1 - resident;
                    if (h == 1) {
                        commit(bars + 2);
                        if (!mbar_wait(bars + 2, ph3)) atomicExch(&g_wide_error, 1);
                        ph3 ^= 1u;
                        mbar_expect_tx(bars + 2, kW3Half);
                        bulk_g2s(sW3, w3img + (size_t)half * kW3Half, kW3Half, bars + 2);
                        if (!mbar_wait(bars + 2, ph3)) atomicExch(&g_wide_error, 1);
                        ph3 ^= 1u;
                        fence_after();
                    }
                    const uint32_t id = idesc_bf16(128, false, false);
#pragma unroll 4
                    for (int k = 0; k < kW2 / 16; ++k)
                        mma(tbase + kTZ + 128 * half, kdesc_at(a0, kW2, 0, 16 * k), kdesc_at(w3, kW2, 0, 16 * k), id,
                            k > 0);
                }
                resident = 1 - resident;
            }
            commit(bars);
            if (TRAIN) {
                bulk_s2g(blob + kBH2, sA, sbuf_bytes(kRows, kW2));
                bulk_commit();
                bulk_wait_read_all();       // H2's region is rewritten by E3
            }
        }
        if (!(ok = wide_wait(bars, ph))) break;
        // E3: logits -> argmax / probabilities (inference) or the cross-entropy and dz (training);
        // the parts' statistics combine in column order
        {
            const int t = TRAIN && valid ? a.target[p] : -1;
            xch[part * kRows + row] = part_lse(tl + kTZ, b3s, zc0, zc1, ncb, t);
            __syncthreads();
            float m = -INFINITY, ssum = 0.f, zt = 0.f;
            int am = 0;
#pragma unroll
            for (int q = 0; q < kParts; ++q) {
                const float4 o = xch[q * kRows + row];
                if (o.x == -INFINITY) continue;               // a part without columns
                const float mn = fmaxf(m, o.x);
                ssum = (m == -INFINITY ? 0.f : ssum * __expf(m - mn)) + o.y * __expf(o.x - mn);
                if (o.x > m) am = __float_as_int(o.z);
                m = mn;
                zt += o.w;                                    // only the part holding the target has it
            }
            const float lse = m + __logf(ssum);
            if (!TRAIN) {
                if (part == 0 && valid && a.argmax) a.argmax[p] = am;
                if (a.prob) {
                    float v[16];
#pragma unroll 1
                    for (int c = zc0; c < zc1 && c < ncb; c += 16) {
                        tmem_ld16(tl + kTZ + c, v);      // every lane: the load is warp-collective
                        if (valid)
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                a.prob[(size_t)(c + j) * a.P + p] = __expf(v[j] + b3s[c + j] - lse);
                    }
                }
            } else {
                const float u = valid ? a.unc[p] : 0.f;
                const float ce = valid ? lse - zt : 0.f;
                const float g = valid ? a.lambda_ce * (1.f - u) : 0.f;
                if (part == 0) {
                    if (valid) a.d_unc[p] = (a.lambda_u - a.lambda_ce * ce) * a.invP;
                    lce += ce * (1.f - u) * a.invP;
                    lu += u * a.invP;
                }
                float v[16];
#pragma unroll 1
                for (int c = zc0; c < zc1; c += 16) {
                    if (c < ncb) tmem_ld16(tl + kTZ + c, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        v[j] = c + j < ncb ? g * (__expf(v[j] + b3s[c + j] - lse) - (c + j == t ? 1.f : 0.f)) : 0.f;
                    sts_bf16x8(smem_u32(sA) + sbuf_off(row, c, 128), v);
                    sts_bf16x8(smem_u32(sA) + sbuf_off(row, c + 8, 128), v + 8);
                }
            }
        }
        if (!TRAIN) {
            fence_before();
            __syncthreads();     // every TMEM read and exchange of this tile before the next tile's MMAs
            fence_after();
            continue;
        }
        cta_publish();
        if (tid == 0) {
            // S4: dh2 = dz W3 (K = ncb; W3 read MN-major)
            const uint32_t a0 = smem_u32(sA), w3 = smem_u32(sW3);
            for (int k = 0; k < ncb / 16; ++k)
                mma(tbase + kTH, kdesc_at(a0, 128, 0, 16 * k), mndesc_at(w3, kW2, 16 * k, 0),
                    idesc_bf16(kW2, false, true), k > 0);
            commit(bars);
            bulk_s2g(blob + kBZ, sA, sbuf_bytes(kRows, 128));
            bulk_commit();
            bulk_wait_read_all();
        }
        if (!(ok = wide_wait(bars, ph))) break;
        // E4: dH2 = dh2 * [h2 > 0]
        mask_epilogue<kW2>(tl + kTH, m2, sA, row, h2c0, h2c1);
        cta_publish();
        if (tid == 0) {
            // S5: dh1 = dH2 W2 (K = 256; W2 read MN-major)
            const uint32_t a0 = smem_u32(sA), w2 = smem_u32(sW2);
#pragma unroll 4
            for (int k = 0; k < kW2 / 16; ++k)
                mma(tbase + kTH, kdesc_at(a0, kW2, 0, 16 * k), mndesc_at(w2, kW1, 16 * k, 0),
                    idesc_bf16(kW1, false, true), k > 0);
            commit(bars);
            bulk_s2g(blob + kBD2, sA, sbuf_bytes(kRows, kW2));
            bulk_commit();
            bulk_wait_read_all();
        }
        if (!(ok = wide_wait(bars, ph))) break;
        // E5: dH1 = dh1 * [h1 > 0]
        mask_epilogue<kW1>(tl + kTH, m1, sA, row, h1c0, h1c1);
        cta_publish();
        if (tid == 0) {
            // S6: dx = dH1 W1 (K = 128; W1 read MN-major), into the logits' columns
            const uint32_t a0 = smem_u32(sA), w1 = smem_u32(sW1);
#pragma unroll
            for (int k = 0; k < kW1 / 16; ++k)
                mma(tbase + kTZ, kdesc_at(a0, kW1, 0, 16 * k), mndesc_at(w1, 16, 16 * k, 0),
                    idesc_bf16(16, false, true), k > 0);
            commit(bars);
            bulk_s2g(blob + kBD1, sA, sbuf_bytes(kRows, kW1));
            bulk_commit();
            bulk_wait_read_all();
        }
        if (!(ok = wide_wait(bars, ph))) break;
        // E6: dL/dR_s
        if (part == 0) {
            float v[16];
            tmem_ld16(tl + kTZ, v);
            if (valid)
#pragma unroll
                for (int c = 0; c < 8; ++c) a.d_feat[(size_t)c * a.P + p] = v[c] * a.invP;
        }
        fence_before();
        __syncthreads();
        fence_after();
    }
    if (TRAIN) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lce += __shfl_xor_sync(0xffffffffu, lce, o);
            lu += __shfl_xor_sync(0xffffffffu, lu, o);
        }
        if (part == 0 && (tid & 31) == 0) {
            atomicAdd(a.loss, lce);
            atomicAdd(a.loss + 1, lu);
        }
        if (tid == 0) bulk_wait_all();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (tid < 32) tmem_dealloc(tbase, 512);
}

// ---------------------------------------------------------------------------
// Pass 2: weight and bias gradients, sum over pixels of outer products of the
// images pass 1 wrote.  blockIdx.y selects the output: 0 -> dW3 [ncb x 256]
// and db3 (A = dZ^T, B = H2 | ones), 1 -> dW2 [256 x 128] and db2 (A = dH2^T
// in two 128-row halves, B = H1 | ones), 2 -> dW1 [128 x 8] and db1 (A =
// dH1^T, B = X, whose column 8 is one).  Every operand is read MN-major:
// the images are pixel-major, and the pixels are the contraction.  Four stages
// of bulk copies, each half a tile (64 pixel rows: the first or second half of
// every image's bytes in the canonical layout), feed the MMAs, so three are in
// flight while one is contracted.
struct WgradArgs {
    int ntiles, ncb;
    float invP;
    const unsigned char* blobs;
    float *dW1, *db1, *dW2, *db2, *dW3, *db3;
};

constexpr int kWStages = 4;
constexpr uint32_t kStage = (sbuf_bytes(kRows, 128) + sbuf_bytes(kRows, kW2)) / 2;   // 48 KB: half a tile
constexpr uint32_t kGOnes = kWStages * kStage, kGBar = kGOnes + sbuf_bytes(kRows, 16),
                   kGSlot = kGBar + 2 * kWStages * 8, kGSmem = kGSlot + 16;

__device__ __forceinline__ void role_parts(int role, uint32_t& off0, uint32_t& n0, uint32_t& off1, uint32_t& n1)
{
    if (role == 0) {
        off0 = kBZ; n0 = sbuf_bytes(kRows, 128); off1 = kBH2; n1 = sbuf_bytes(kRows, kW2);
    } else if (role == 1) {
        off0 = kBD2; n0 = sbuf_bytes(kRows, kW2); off1 = kBH1; n1 = sbuf_bytes(kRows, kW1);
    } else {
        off0 = kBD1; n0 = sbuf_bytes(kRows, kW1); off1 = kBX; n1 = kXBytes;
    }
}

__global__ void __launch_bounds__(kRows, 1) wide_wgrad_kernel(WgradArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* const ones = sm + kGOnes;
    uint64_t* const full = reinterpret_cast<uint64_t*>(sm + kGBar);     // [kWStages]
    uint64_t* const empty = full + kWStages;                            // [kWStages]
    uint32_t* const slot = reinterpret_cast<uint32_t*>(sm + kGSlot);
    const int tid = threadIdx.x, role = blockIdx.y;
    uint32_t off0, n0, off1, n1;
    role_parts(role, off0, n0, off1, n1);
    {
        float v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = c == 0 ? 1.f : 0.f;
        sbuf_store8(SBuf{ones, 16}, tid, 0, v);
        sbuf_store8(SBuf{ones, 16}, tid, 8, v + 8);
    }
    if (tid == 0)
        for (int k = 0; k < 2 * kWStages; ++k) mbar_init(full + k, 1);
    if (tid < 32) tmem_alloc(slot, 512);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(slot);
    // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int n = a.ntiles > (int)blockIdx.x ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    bool ok = true;
    if (tid == 0) {
        // half-tile q = 2 i + hf of this CTA's i-th tile goes through stage q % kWStages
        const uint32_t h0 = n0 / 2, h1 = n1 / 2;
        auto load = [&](int q) {
            const int st = q % kWStages, hf = q & 1;
            const unsigned char* b = a.blobs + (size_t)((int)blockIdx.x + (q >> 1) * (int)gridDim.x) * kBlob;
            mbar_expect_tx(full + st, h0 + h1);
            bulk_g2s(sm + st * kStage, b + off0 + hf * h0, h0, full + st);
            bulk_g2s(sm + st * kStage + h0, b + off1 + hf * h1, h1, full + st);
        };
        const int nq = 2 * n;
        for (int q = 0; q < kWStages && q < nq; ++q) load(q);
        const uint32_t on = smem_u32(ones);
        for (int q = 0; q < nq && ok; ++q) {
            const int st = q % kWStages;
            if (!mbar_wait(full + st, (uint32_t)(q / kWStages) & 1u)) {
                ok = false;
                break;
            }
            fence_after();
            const uint32_t p0 = smem_u32(sm + st * kStage), p1 = p0 + h0;
#pragma unroll 1
            for (int k = 0; k < kRows / 32; ++k) {
                const uint32_t acc = q > 0 || k > 0;
                if (role == 0) {
                    const uint64_t A = mndesc_at(p0, 128, 16 * k, 0);
                    mma(tbase, A, mndesc_at(p1, kW2, 16 * k, 0), idesc_bf16(kW2, true, true), acc);
                    mma(tbase + 256, A, mndesc_at(on, 16, 16 * k, 0), idesc_bf16(16, true, true), acc);
                } else if (role == 1) {
                    const uint64_t B = mndesc_at(p1, kW1, 16 * k, 0), O = mndesc_at(on, 16, 16 * k, 0);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint64_t A = mndesc_at(p0, kW2, 16 * k, 128 * h);
                        mma(tbase + 128 * h, A, B, idesc_bf16(kW1, true, true), acc);
                        mma(tbase + 256 + 16 * h, A, O, idesc_bf16(16, true, true), acc);
                    }
                } else {
                    mma(tbase, mndesc_at(p0, kW1, 16 * k, 0), mndesc_at(p1, 16, 16 * k, 0),
                        idesc_bf16(16, true, true), acc);
                }
            }
            commit(empty + st);
            // refill the stage of half-tile q - 1 with half-tile q - 1 + kWStages
            if (q >= 1 && q - 1 + kWStages < nq) {
                const int sp = (q - 1) % kWStages;
                if (!mbar_wait(empty + sp, (uint32_t)((q - 1) / kWStages) & 1u)) {
                    ok = false;
                    break;
                }
                load(q - 1 + kWStages);
            }
        }
        // the last half-tile's MMAs
        if (ok && nq > 0 && !mbar_wait(empty + (nq - 1) % kWStages, (uint32_t)((nq - 1) / kWStages) & 1u))
            ok = false;
        if (!ok) atomicExch(&g_wide_error, 1);
    }
    const bool bad = bar_any(0, kRows, !ok);
    fence_after();
    if (!bad && n > 0) {
        const uint32_t tl = tbase + ((uint32_t)(32 * (tid >> 5)) << 16);
        float v[16];
        if (role == 0) {
            // row = code; the loads are warp-collective, the codes past ncb add nothing
#pragma unroll 1
            for (int c = 0; c < kW2; c += 16) {
                tmem_ld16(tl + c, v);
                if (tid < a.ncb)
#pragma unroll
                    for (int j = 0; j < 16; ++j) atomicAdd(a.dW3 + (size_t)tid * kW2 + c + j, v[j] * a.invP);
            }
            tmem_ld16(tl + 256, v);
            if (tid < a.ncb) atomicAdd(a.db3 + tid, v[0] * a.invP);
        } else if (role == 1) {
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                const int r = 128 * h + tid;
#pragma unroll 1
                for (int c = 0; c < kW1; c += 16) {
                    tmem_ld16(tl + 128 * h + c, v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) atomicAdd(a.dW2 + (size_t)r * kW1 + c + j, v[j] * a.invP);
                }
                tmem_ld16(tl + 256 + 16 * h, v);
                atomicAdd(a.db2 + r, v[0] * a.invP);
            }
        } else {
            tmem_ld16(tl, v);
#pragma unroll
            for (int c = 0; c < 8; ++c) atomicAdd(a.dW1 + (size_t)tid * 8 + c, v[c] * a.invP);
            atomicAdd(a.db1 + tid, v[8] * a.invP);
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (tid < 32) tmem_dealloc(tbase, 512);
}

// FP32 weights [out][in] -> the BF16 canonical images: W1 [128 x 16] (inputs
// 8..15 zero), W2 [256 x 128], W3 [R x 256] (R = ncb, or 256 with the codes
// past ncb zero when W3 takes two halves).
__global__ void wide_images_kernel(const float* __restrict__ W1, const float* __restrict__ W2,
                                   const float* __restrict__ W3, int ncb, int r3, unsigned char* __restrict__ img)
{
    const int n1 = kW1 * 2, n2 = kW2 * (kW1 / 8), n3 = r3 * (kW2 / 8);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2 + n3; i += gridDim.x * blockDim.x) {
        float v[8];
        if (i < n1) {
            const int r = i / 2, c0 = (i % 2) * 8;
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = c0 + j < 8 ? W1[r * 8 + c0 + j] : 0.f;
            sbuf_store8(SBuf{img, 16}, r, c0, v);
        } else if (i < n1 + n2) {
            const int k = i - n1, r = k / (kW1 / 8), c0 = (k % (kW1 / 8)) * 8;
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = W2[(size_t)r * kW1 + c0 + j];
            sbuf_store8(SBuf{img + kW1Bytes, kW1}, r, c0, v);
        } else {
            const int k = i - n1 - n2, r = k / (kW2 / 8), c0 = (k % (kW2 / 8)) * 8;
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = r < ncb ? W3[(size_t)r * kW2 + c0 + j] : 0.f;
            sbuf_store8(SBuf{img + kW1Bytes + kW2Bytes, kW2}, r, c0, v);
        }
    }
}

int wide_sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        n = 1;
    return n;
}

size_t images_bytes(int ncb) { return align_up(kW1Bytes + kW2Bytes + (ncb > 128 ? 2 * kW3Half : (size_t)ncb * kW2 * 2), 256); }

}  // namespace

bool wide_decoder(const le_decoder* d) { return d->d_in == 8 && d->h1 == kW1 && d->h2 == kW2; }

le_status check_wide_decoder(const le_decoder* d, bool train)
{
    if (!wide_decoder(d) || d->n_cb % 16 != 0 || d->n_cb < 16 || d->n_cb > (train ? 128 : 256)) {
        set_error("the tensor-core path at the widths 8-128-256-N supports n_cb a multiple of 16 in [16, %d]; got %d",
                  train ? 128 : 256, d->n_cb);
        return LE_ERR_UNSUPPORTED;
    }
    return LE_OK;
}

size_t wide_workspace(int32_t P, const le_decoder* d, bool train)
{
    const size_t nt = ((size_t)P + kRows - 1) / kRows;
    return images_bytes(d->n_cb) + (train ? nt * kBlob : 0);
}

le_status wide_decode(int32_t P, const float* feat, const float* unc, const le_decoder* d, const int32_t* target,
                      float lambda_ce, float lambda_u, float* loss, float* d_feat, float* d_unc,
                      const le_decoder_grads* dg, int32_t* argmax, float* prob, void* ws, size_t ws_bytes,
                      cudaStream_t s)
{
    const bool train = target != nullptr;
    le_status st = check_wide_decoder(d, train);
    if (st != LE_OK) return st;
    const int ncb = d->n_cb;
    LE_CHECK_ARG(ws && (reinterpret_cast<uintptr_t>(ws) & 255u) == 0 && ws_bytes >= wide_workspace(P, d, train),
                 "workspace must be 256-byte aligned and at least %zu bytes", wide_workspace(P, d, train));
    unsigned char* img = static_cast<unsigned char*>(ws);
    wide_images_kernel<<<64, 256, 0, s>>>(d->W1, d->W2, d->W3, ncb, ncb > 128 ? 256 : ncb, img);
    LE_LAUNCHED();
    WideArgs a{};
    a.P = P;
    a.ncb = ncb;
    a.feat = feat;
    a.unc = unc;
    a.target = target;
    a.b1 = d->b1; a.b2 = d->b2; a.b3 = d->b3;
    a.img = img;
    a.lambda_ce = lambda_ce;
    a.lambda_u = lambda_u;
    a.invP = 1.0f / (float)P;
    a.loss = loss;
    a.d_feat = d_feat;
    a.d_unc = d_unc;
    a.argmax = argmax;
    a.prob = prob;
    a.blobs = img + images_bytes(ncb);
    const int ntiles = (P + kRows - 1) / kRows;
    const int sms = wide_sm_count();
    const int grid = ntiles < sms ? ntiles : sms;
    if (!train) {
        LE_CUDA(cudaFuncSetAttribute(wide_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
        wide_kernel<false><<<grid, kThreads, kSmem, s>>>(a);
        LE_LAUNCHED();
        return LE_OK;
    }
    LE_CUDA(cudaMemsetAsync(loss, 0, 2 * sizeof(float), s));
    LE_CUDA(cudaMemsetAsync(dg->W1, 0, sizeof(float) * kW1 * 8, s));
    LE_CUDA(cudaMemsetAsync(dg->b1, 0, sizeof(float) * kW1, s));
    LE_CUDA(cudaMemsetAsync(dg->W2, 0, sizeof(float) * kW2 * kW1, s));
    LE_CUDA(cudaMemsetAsync(dg->b2, 0, sizeof(float) * kW2, s));
    LE_CUDA(cudaMemsetAsync(dg->W3, 0, sizeof(float) * ncb * kW2, s));
    LE_CUDA(cudaMemsetAsync(dg->b3, 0, sizeof(float) * ncb, s));
    LE_CUDA(cudaFuncSetAttribute(wide_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    wide_kernel<true><<<grid, kThreads, kSmem, s>>>(a);
    LE_LAUNCHED();
    WgradArgs g{};
    g.ntiles = ntiles;
    g.ncb = ncb;
    g.invP = a.invP;
    g.blobs = a.blobs;
    g.dW1 = dg->W1; g.db1 = dg->b1; g.dW2 = dg->W2; g.db2 = dg->b2; g.dW3 = dg->W3; g.db3 = dg->b3;
    const int slices = ntiles < sms / 3 ? ntiles : (sms / 3 > 0 ? sms / 3 : 1);
    LE_CUDA(cudaFuncSetAttribute(wide_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmem));
    wide_wgrad_kernel<<<dim3(slices, 3), kRows, kGSmem, s>>>(g);
    LE_LAUNCHED();
    return LE_OK;
}

le_status wide_take_timeout(bool* timed_out)
{
    int flag = 0;
    LE_CUDA(cudaMemcpyFromSymbol(&flag, g_wide_error, sizeof(int)));
    *timed_out = flag != 0;
    if (flag) {
        const int zero = 0;
        LE_CUDA(cudaMemcpyToSymbol(g_wide_error, &zero, sizeof(int)));
    }
    return LE_OK;
}

}  // namespace leg
