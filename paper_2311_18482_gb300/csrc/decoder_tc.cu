// Fused semantic decoder on the 5th-generation tensor cores (tcgen05, BF16
// operands, FP32 accumulation in TMEM).
//
// D_MLP (Eq. 8, eq:lem_dec; supp. Tab. dmlp, here 8 -> 64 -> 128 -> N) runs per
// 128-pixel tile: the rendered feature R_s of the tile is the A operand of
// three chained MMAs whose accumulators never leave the SM; the CUDA cores
// only apply bias + ReLU between layers (TMEM -> registers -> BF16 shared
// memory) and the softmax at the end.  Three kernels share that front end:
//
//   dec_fwd_kernel    inference (supp. Sec. "Inference"): argmax and/or
//                     M_infer = softmax(logits), two tiles in flight per CTA.
//   dec_train_kernel  training step (Eqs. 9-12): uncertainty-weighted CE,
//                     dL/dR_u, and the whole backward on the tensor cores,
//                     warp-specialised with two tiles in flight (one MMA
//                     warp, four epilogue warpgroups).  dL/dz, dL/dh2 and
//                     dL/dh1 are written once, pixel-major; the input-gradient
//                     MMAs read them K-major and the weight-gradient MMAs read
//                     the same buffers MN-major (contracting over the tile's
//                     pixels); bias gradients are MMAs against a ones operand.
//                     Weight gradients accumulate in TMEM over all tiles of a
//                     CTA and are flushed once.
//   query_fused_kernel relevancy (supp. Sec. "Inference", LERF): with
//                     p proportional to e = exp(z - max z), |F_clip|^2 =
//                     p^T (S_c S_c^T) p and phi.q_j = p.(S_c q_j)/|F_clip|; the
//                     relevancy does not depend on the scale of p, so neither
//                     the softmax normaliser nor the 896-dim feature map F is
//                     ever formed; S_c S_c^T (N x N) is streamed through shared
//                     memory in 64-column chunks with 1-D bulk async copies,
//                     S_c [q; n] sits in shared memory.
//
// Every mbarrier wait is bounded (about a second); on timeout the kernel
// records it in g_tc_error, stops issuing work, frees its TMEM and returns.
#include "tc_common.cuh"

namespace leg {

__device__ int g_tc_error;

namespace {
using namespace tc;

constexpr int kD = 8, kH1 = 64, kH2 = 128;

struct DecArgs {
    int P, ncb;
    const float *feat, *unc;
    const int32_t* target;
    const float *W1, *b1, *W2, *b2, *W3, *b3;
    float lambda_ce, lambda_u, invP;
    float* loss;
    float *d_feat, *d_unc;
    float *dW1, *db1, *dW2, *db2, *dW3, *db3;
    int32_t* argmax;
    float* prob;
    // feature-map export: W3 as the BF16 shared-memory image (reloaded per tile
    // when the output staging borrows W3's shared memory)
    const unsigned char* W3_img;
    int w3_reload;
    // query
    const unsigned char* G_img;     // ncb/64 chunks of [ncb x 64] canonical bf16
    const float* Aq;                // [16, ncb] fp32 = [text; negs] S_c^T
    int Q, n_neg;
    float* rel;
    // feature-map export
    int dd;                         // feature dims d (multiple of 64)
    __nv_bfloat16* fmap;            // [P, dd] out
    // training with the RGB L1 term of the same pixels (nullable img): img, img_t [3, P],
    // d_img [3, P] = sign(img - img_t) inv_l1, *loss_l1 += sum |img - img_t| inv_l1
    const float *img, *img_t;
    float *d_img, *loss_l1;
    float inv_l1;
};

// Per-warpgroup state of the shared MLP front end.  With nhalf = 2 or 4,
// that many warpgroups serve the same 128 TMEM lanes (rows) and split every
// epilogue by columns; `xch` is their shared-memory exchange for row-wide
// statistics ([nhalf][128] float4).
struct Front {
    SBuf W1s, W2s, W3s, X1, H1, H2;
    const float *b1s, *b2s, *b3s;
    uint64_t* mbar;
    uint32_t phase;
    uint32_t tw;       // TMEM column base of this warpgroup's working accumulator
    uint32_t lane;     // this warp's TMEM lane field
    int tid;           // row of the tile (TMEM lane) this thread serves
    int bar_id, nthreads;
    int half, nhalf;
    float4* xch;       // [nhalf][128] (nhalf > 1 only)
    // W3s reloaded by a bulk copy (thread 0 only): the third layer's MMAs wait
    // for it first
    uint64_t* w3bar = nullptr;
    uint32_t w3phase = 0;
    bool w3pending = false;
};

// Columns [c0, c1) of an N-column epilogue handled by this thread's half (units of 16).
__device__ __forceinline__ void my_cols(const Front& f, int N, int& c0, int& c1)
{
    const int nch = N / 16, per = (nch + f.nhalf - 1) / f.nhalf;
    c0 = min(nch, f.half * per) * 16;
    c1 = min(nch, (f.half + 1) * per) * 16;
}

__device__ __forceinline__ void wg_sync(const Front& f)
{
    if (f.nthreads == (int)blockDim.x) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(f.bar_id), "r"(f.nthreads) : "memory");
}

// Wait for this warpgroup's MMA barrier; false (for every thread) if any thread timed out.
__device__ __forceinline__ bool wg_wait(Front& f)
{
    const bool ok = mbar_wait(f.mbar, f.phase);
    f.phase ^= 1u;
    const bool bad = bar_any(f.bar_id, f.nthreads, !ok);
    if (bad && f.tid == 0) atomicExch(&g_tc_error, 1);
    fence_after();
    return !bad;
}

// Make this warpgroup's shared-memory writes visible to the tensor core and
// order them (and all TMEM reads) before the MMAs issued next.
__device__ __forceinline__ void wg_publish(const Front& f)
{
    fence_proxy_async();
    fence_before();
    wg_sync(f);
    fence_after();
}

// D_MLP forward of one 128-pixel tile: X1 <- feat (col 8 = 1 for the bias
// gradient), H1 = relu(W1 x + b1), H2 = relu(W2 h1 + b2), logits - b3 left in
// TMEM columns [tw, tw + ncb).  Returns false on a timed-out wait.
// R_s of pixel p (zeros past the end), for mlp_forward_x.
__device__ __forceinline__ void load_feat(const DecArgs& a, int p, bool valid, float* x)
{
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = valid ? a.feat[(size_t)c * a.P + p] : 0.f;
}

// mlp_forward with the tile's features already in registers (x, read by the
// first part only), so that a caller can load them a tile ahead.
__device__ bool mlp_forward_x(Front& f, const DecArgs& a, const float* x)
{
    float v[16];
    if (f.half == 0) sbuf_store8(f.X1, f.tid, 0, x);
    if (f.half == f.nhalf - 1) {
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = c == 0 ? 1.f : 0.f;
        sbuf_store8(f.X1, f.tid, 8, v);
    }
    wg_publish(f);
    if (f.tid == 0 && f.half == 0) {
        mma(f.tw, kdesc(f.X1, 0, 0), kdesc(f.W1s, 0, 0), idesc_bf16(kH1, false, false), 0);
        commit(f.mbar);
    }
    if (!wg_wait(f)) return false;
    int c0, c1;
    my_cols(f, kH1, c0, c1);
    for (int c = c0; c < c1; c += 16) {
        tmem_ld16(f.tw + f.lane + c, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + f.b1s[c + j], 0.f);
        sbuf_store8(f.H1, f.tid, c, v);
        sbuf_store8(f.H1, f.tid, c + 8, v + 8);
    }
    wg_publish(f);
    if (f.tid == 0 && f.half == 0) {
#pragma unroll
        for (int s = 0; s < kH1 / 16; ++s)
            mma(f.tw, kdesc(f.H1, 0, 16 * s), kdesc(f.W2s, 0, 16 * s), idesc_bf16(kH2, false, false), s > 0);
        commit(f.mbar);
    }
    if (!wg_wait(f)) return false;
    my_cols(f, kH2, c0, c1);
    for (int c = c0; c < c1; c += 16) {
        tmem_ld16(f.tw + f.lane + c, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j] + f.b2s[c + j], 0.f);
        sbuf_store8(f.H2, f.tid, c, v);
        sbuf_store8(f.H2, f.tid, c + 8, v + 8);
    }
    wg_publish(f);
    if (f.tid == 0 && f.half == 0) {
        if (f.w3pending) {
            if (!mbar_wait(f.w3bar, f.w3phase)) atomicExch(&g_tc_error, 1);
            f.w3phase ^= 1u;
            f.w3pending = false;
        }
#pragma unroll
        for (int s = 0; s < kH2 / 16; ++s)
            mma(f.tw, kdesc(f.H2, 0, 16 * s), kdesc(f.W3s, 0, 16 * s), idesc_bf16(a.ncb, false, false), s > 0);
        commit(f.mbar);
    }
    return wg_wait(f);
}

__device__ bool mlp_forward(Front& f, const DecArgs& a, int p, bool valid)
{
    float x[8];
    if (f.half == 0) load_feat(a, p, valid, x);
    return mlp_forward_x(f, a, x);
}

// Online max / argmax / log-sum-exp over the ncb logits in TMEM (+ b3); with
// several parts, each covers its columns and they combine through f.xch in
// column order.  Ties go to the lowest index.  zt = logit of class t (if t >= 0).
__device__ __forceinline__ void logits_lse(const Front& f, int ncb, float& lse, int& am, int t, float& zt)
{
    float m = -INFINITY, s = 0.f, v[16];
    am = 0;
    zt = 0.f;
    int c0, c1;
    my_cols(f, ncb, c0, c1);
    for (int c = c0; c < c1; c += 16) {
        tmem_ld16(f.tw + f.lane + c, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float z = v[j] + f.b3s[c + j];
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
    if (f.nhalf > 1) {
        f.xch[f.half * 128 + f.tid] = make_float4(m, s, __int_as_float(am), zt);
        wg_sync(f);
        float mt = -INFINITY, st = 0.f, zsum = 0.f;
        int at = 0;
        for (int h = 0; h < f.nhalf; ++h) {
            const float4 o = f.xch[h * 128 + f.tid];
            if (o.x == -INFINITY) continue;           // a part without columns
            const float mn = fmaxf(mt, o.x);
            st = (mt == -INFINITY ? 0.f : st * __expf(mt - mn)) + o.y * __expf(o.x - mn);
            if (o.x > mt) at = __float_as_int(o.z);
            mt = mn;
            zsum += o.w;                             // only the part holding class t has it
        }
        wg_sync(f);
        m = mt;
        s = st;
        am = at;
        zt = zsum;
    }
    lse = m + __logf(s);
}

__host__ __device__ constexpr size_t weights_bytes(int ncb)
{
    return (size_t)sbuf_bytes(64, 16) + sbuf_bytes(128, 64) + sbuf_bytes(ncb, 128) +
           ((size_t)(64 + 128 + ncb) * 4 + 127) / 128 * 128;
}

// Carve weights + biases at `base`, fill them (all threads).
__device__ unsigned char* load_weights(unsigned char* base, const DecArgs& a, Front& f)
{
    unsigned char* p = base;
    f.W1s = SBuf{p, 16};
    p += sbuf_bytes(64, 16);
    f.W2s = SBuf{p, 64};
    p += sbuf_bytes(128, 64);
    f.W3s = SBuf{p, 128};
    p += sbuf_bytes(a.ncb, 128);
    float* bs = reinterpret_cast<float*>(p);
    p += ((size_t)(64 + 128 + a.ncb) * 4 + 127) / 128 * 128;
    sbuf_fill(f.W1s, 64, a.W1, kD, 64, kD);
    sbuf_fill(f.W2s, 128, a.W2, kH1, 128, kH1);
    sbuf_fill(f.W3s, a.ncb, a.W3, kH2, a.ncb, kH2);
    for (int i = threadIdx.x; i < 64 + 128 + a.ncb; i += blockDim.x)
        bs[i] = i < 64 ? a.b1[i] : (i < 192 ? a.b2[i - 64] : a.b3[i - 192]);
    f.b1s = bs;
    f.b2s = bs + 64;
    f.b3s = bs + 192;
    return p;
}

// ---------------------------------------------------------------------------
// Inference.  NWG warpgroups per CTA, each with its own tile, buffers,
// mbarrier and 256 TMEM columns; weights shared.
constexpr size_t kFwdWgBytes = sbuf_bytes(128, 16) + sbuf_bytes(128, 64) + sbuf_bytes(128, 128);

__host__ constexpr size_t fwd_smem(int ncb, int nwg) { return weights_bytes(ncb) + nwg * kFwdWgBytes + 128; }

template <int NWG>
__global__ void __launch_bounds__(128 * NWG, 1) dec_fwd_kernel(DecArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    Front f;
    unsigned char* p = load_weights(sm, a, f);
    const int wg = threadIdx.x >> 7;
    unsigned char* q = p + wg * kFwdWgBytes;
    f.X1 = SBuf{q, 16};
    f.H1 = SBuf{q + sbuf_bytes(128, 16), 64};
    f.H2 = SBuf{q + sbuf_bytes(128, 16) + sbuf_bytes(128, 64), 128};
    uint64_t* mbars = reinterpret_cast<uint64_t*>(p + NWG * kFwdWgBytes);
    uint32_t* slot = reinterpret_cast<uint32_t*>(mbars + NWG);
    f.mbar = mbars + wg;
    f.phase = 0;
    f.tid = threadIdx.x & 127;
    f.bar_id = 1 + wg;
    f.nthreads = NWG == 1 ? (int)blockDim.x : 128;
    f.half = 0;
    f.nhalf = 1;
    f.xch = nullptr;
    if (threadIdx.x == 0)
        for (int w = 0; w < NWG; ++w) mbar_init(mbars + w, 1);
    if (threadIdx.x < 32) tmem_alloc(slot, 256 * NWG);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(slot);
    f.tw = tbase + 256 * wg;
    f.lane = (uint32_t)(32 * (f.tid >> 5)) << 16;

    const int ntiles = (a.P + 127) / 128;
    for (int tile = blockIdx.x * NWG + wg; tile < ntiles; tile += gridDim.x * NWG) {
        const int px = tile * 128 + f.tid;
        const bool valid = px < a.P;
        if (!mlp_forward(f, a, px, valid)) break;
        float lse, zt;
        int am;
        logits_lse(f, a.ncb, lse, am, -1, zt);
        if (valid && a.argmax) a.argmax[px] = am;
        if (a.prob) {
            float v[16];
            for (int c = 0; c < a.ncb; c += 16) {
                tmem_ld16(f.tw + f.lane + c, v);
                if (valid)
#pragma unroll
                    for (int j = 0; j < 16; ++j) a.prob[(size_t)(c + j) * a.P + px] = __expf(v[j] + f.b3s[c + j] - lse);
            }
        }
        fence_before();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tbase, 256 * NWG);
}

// ---------------------------------------------------------------------------
// Training.  One CTA per SM, persistent over tiles and warp-specialised: warp
// 16 issues every MMA; warpgroups 0-3 run the epilogues of two tiles in flight
// (slot s = warpgroups 2s and 2s+1, which serve the same 128 rows and split
// every epilogue by columns), so the tensor core works on one slot while the
// CUDA cores finish the other.  Per tile, six MMA stages alternate with six
// epilogues (z = logits, dz = dL/dz etc.):
//   S1  h1 = X1 W1^T                                E1  bias, ReLU -> H1; ReLU mask kept in registers
//   S2  h2 = H1 W2^T                                E2  bias, ReLU -> H2; mask
//   S3  z  = H2 W3^T                                E3  softmax, CE (Eqs. 9-12) -> dz into D
//   S4  dh2 = dz W3;  dW3 += dz^T h2;  db3 += dz^T 1   E4  mask -> dh2 into H2's buffer
//   S5  dh1 = dh2 W2; dW2 += dh2^T h1; db2 += dh2^T 1  E5  mask -> dh1 into D
//   S6  dx  = dh1 W1; [dW1 | db1] += dh1^T [x | 1]     E6  dx -> d_feat
// dz, dh2 and dh1 are stored pixel-major: the input-gradient MMAs read them
// K-major and the weight-gradient MMAs MN-major (contracting over the tile's
// pixels).  Handshake per slot: its 256 epilogue threads arrive on ready[s]
// once their operand is in shared memory and their TMEM reads are done; the
// MMA thread waits, issues, and commits to done[s].  All MMAs come from one
// thread, so the weight-gradient accumulations of both slots are ordered.
// TMEM (512 columns): working accumulators [0,128) and [128,256); dW3
// [256,384); dW2 [384,448); block P [448,464) holds db2 (column 0, again in 9)
// and db3 (column 8); block Q [480,496) holds dW1 (columns 0-7) and db1 (8).
// The ones operand E (128 pixels x 24, ones in columns 8 and 17) read from
// column 0 sums over pixels into output column 8, read from column 8 into
// columns 0 and 9 -- so db3 and db2 share block P without overlapping.
constexpr int kTrainThreads = 4 * 128 + 32;
constexpr uint32_t kTW3 = 256, kTW2 = 384, kTP = 448, kTQ = 480;
constexpr int kEC = 24;

// Shared-memory addresses of one slot's buffers (column counts 16, 64, 128, 128):
// X1; H1; H2, later dh2; D: dz (and the softmax exchange), later dh1.
constexpr uint32_t kSX1 = 0, kSH1 = sbuf_bytes(128, 16), kSH2 = kSH1 + sbuf_bytes(128, kH1),
                   kSD = kSH2 + sbuf_bytes(128, 128), kSlotBytes = kSD + sbuf_bytes(128, 128);

__host__ __device__ constexpr size_t train_slot_bytes() { return kSlotBytes; }

__host__ constexpr size_t train_smem(int ncb)
{
    return weights_bytes(ncb) + sbuf_bytes(128, kEC) + 2 * train_slot_bytes() + 128;
}

// Issue MMA stage `st` (0-5) of the slot whose buffers start at shared address
// q.  `init`: the first tile of this CTA, whose weight-gradient MMAs overwrite
// their accumulators.  Each operand's descriptor is built once per stage; the
// next 16-wide K step only moves the start address, by 16 (K-major: one pair
// of core matrices, 256 B) or by 2C (MN-major over a C-column buffer: two
// 8-row groups, 32 C bytes) in descriptor units of 16 B.
__device__ __forceinline__ void train_stage(int st, int ncb, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t e,
                                            uint32_t q, uint32_t tw, uint32_t tb, bool init)
{
    const uint32_t keep = init ? 0u : 1u;
    const uint32_t x1 = q + kSX1, h1 = q + kSH1, h2 = q + kSH2, d = q + kSD;
    switch (st) {
        case 0:
            mma(tw, kdesc_at(x1, 16, 0, 0), kdesc_at(w1, 16, 0, 0), idesc_bf16(kH1, false, false), 0);
            break;
        case 1: {
            const uint64_t a = kdesc_at(h1, kH1, 0, 0), b = kdesc_at(w2, kH1, 0, 0);
#pragma unroll
            for (int k = 0; k < kH1 / 16; ++k) mma(tw, a + 16 * k, b + 16 * k, idesc_bf16(kH2, false, false), k > 0);
            break;
        }
        case 2: {
            const uint64_t a = kdesc_at(h2, 128, 0, 0), b = kdesc_at(w3, 128, 0, 0);
            const uint32_t id = idesc_bf16(ncb, false, false);
#pragma unroll
            for (int k = 0; k < kH2 / 16; ++k) mma(tw, a + 16 * k, b + 16 * k, id, k > 0);
            break;
        }
        case 3: {
            const uint64_t ak = kdesc_at(d, 128, 0, 0), w3m = mndesc_at(w3, 128, 0, 0);
            for (int k = 0; k < ncb / 16; ++k)
                mma(tw, ak + 16 * k, w3m + 256 * k, idesc_bf16(kH2, false, true), k > 0);
            const uint64_t am = mndesc_at(d, 128, 0, 0), h2m = mndesc_at(h2, 128, 0, 0), em = mndesc_at(e, kEC, 0, 0);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                mma(tb + kTW3, am + 256 * k, h2m + 256 * k, idesc_bf16(kH2, true, true), k > 0 ? 1u : keep);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                mma(tb + kTP, am + 256 * k, em + 2 * kEC * k, idesc_bf16(16, true, true), k > 0 ? 1u : keep);
            break;
        }
        case 4: {
            const uint64_t ak = kdesc_at(h2, 128, 0, 0), w2m = mndesc_at(w2, kH1, 0, 0);
#pragma unroll
            for (int k = 0; k < kH2 / 16; ++k)
                mma(tw, ak + 16 * k, w2m + 2 * kH1 * k, idesc_bf16(kH1, false, true), k > 0);
            const uint64_t am = mndesc_at(h2, 128, 0, 0), h1m = mndesc_at(h1, kH1, 0, 0),
                           em = mndesc_at(e, kEC, 0, 8);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                mma(tb + kTW2, am + 256 * k, h1m + 2 * kH1 * k, idesc_bf16(kH1, true, true), k > 0 ? 1u : keep);
#pragma unroll
            for (int k = 0; k < 8; ++k) mma(tb + kTP, am + 256 * k, em + 2 * kEC * k, idesc_bf16(16, true, true), 1u);
            break;
        }
        default: {
            const uint64_t ak = kdesc_at(d, 128, 0, 0), w1m = mndesc_at(w1, 16, 0, 0);
#pragma unroll
            for (int k = 0; k < kH1 / 16; ++k)
                mma(tw, ak + 16 * k, w1m + 2 * 16 * k, idesc_bf16(16, false, true), k > 0);
            const uint64_t am = mndesc_at(d, 128, 0, 0), x1m = mndesc_at(x1, 16, 0, 0);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                mma(tb + kTQ, am + 256 * k, x1m + 2 * 16 * k, idesc_bf16(16, true, true), k > 0 ? 1u : keep);
            break;
        }
    }
}

// The MMA thread: tile pairs in order, stage by stage, slot 0 then slot 1.
__device__ __forceinline__ bool train_mma_loop(int ncb, const Front& f, uint32_t e, uint32_t slots,
                                               uint64_t* ready, uint64_t* done, uint32_t tb, int ntiles)
{
    uint32_t ph[2] = {0u, 0u};
    const uint32_t w1 = smem_u32(f.W1s.p), w2 = smem_u32(f.W2s.p), w3 = smem_u32(f.W3s.p);
    for (int it = 0;; ++it) {
        const int t0 = blockIdx.x + 2 * it * gridDim.x;
        if (t0 >= ntiles) break;
        const int nsl = t0 + (int)gridDim.x < ntiles ? 2 : 1;
        for (int st = 0; st < 6; ++st)
            for (int s = 0; s < nsl; ++s) {
                if (!mbar_wait(ready + s, ph[s])) return false;
                ph[s] ^= 1u;
                fence_after();
                train_stage(st, ncb, opaque(w1), opaque(w2), opaque(w3), opaque(e), opaque(slots + kSlotBytes * s),
                            tb + 128u * s, tb, it == 0 && s == 0);
                commit(done + s);
            }
    }
    return true;
}

// Epilogue thread state: slot s (buffers at shared address sb), half h of the
// columns, tile row `row`.
struct EpiCtx {
    uint32_t sb;
    uint64_t *ready, *done;
    uint32_t tw, lanef, ph;
    int s, h, row, bar_id;
};

__device__ __forceinline__ void epi_signal(const EpiCtx& e)
{
    fence_proxy_async();
    fence_before();
    mbar_arrive(e.ready);
}

// Wait for the slot's MMAs; the outcome is made uniform over the slot's 256
// threads, so a timeout never leaves part of them at the exchange barrier.
__device__ __forceinline__ bool epi_wait(EpiCtx& e)
{
    const bool ok = !bar_any(e.bar_id, 256, !mbar_wait(e.done, e.ph));
    e.ph ^= 1u;
    fence_after();
    return ok;
}

// Byte offset of exchange entry i (0-255) in the 128-column canonical buffer D:
// the 16-byte chunk (row 8 (i/16) + i%8, columns 8 ((i/8)%2) ...), i.e. every
// entry lies in columns [0, 16).
__device__ __forceinline__ uint32_t xch_off(int i)
{
    return (uint32_t)((i >> 4) * 2048 + ((i >> 3) & 1) * 128 + (i & 7) * 16);
}

__device__ __forceinline__ float4 ld_bias4(const float* b, int c) { return *reinterpret_cast<const float4*>(b + c); }

// bias + ReLU over 16 columns starting at c: v <- relu(v + b); bit j of the
// result = (v_j > 0)
__device__ __forceinline__ uint32_t bias_relu16(float* v, const float* b, int c)
{
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < 16; j += 4) {
        const float4 bb = ld_bias4(b, c + j);
        const float bj[4] = {bb.x, bb.y, bb.z, bb.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float x = v[j + i] + bj[i];
            m |= (x > 0.f ? 1u : 0u) << (j + i);
            v[j + i] = fmaxf(x, 0.f);
        }
    }
    return m;
}

__device__ __forceinline__ void mask16(float* v, uint32_t m)
{
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = (m >> j) & 1u ? v[j] : 0.f;
}

// 16 columns [c, c + 16) of row `row` of the C-column buffer at shared address b.
__device__ __forceinline__ void store16(uint32_t b, int C, int row, int c, const float* v)
{
    sts_bf16x8(b + sbuf_off(row, c, C), v);
    sts_bf16x8(b + sbuf_off(row, c + 8, C), v + 8);
}

// v[idx] for a runtime idx in [0, 16), by a select tree over the index bits
// (keeps v in registers).
__device__ __forceinline__ float select16(const float* v, int idx)
{
    float t8[8], t4[4], t2[2];
    const bool b0 = idx & 1, b1 = idx & 2, b2 = idx & 4, b3 = idx & 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) t8[i] = b0 ? v[2 * i + 1] : v[2 * i];
#pragma unroll
    for (int i = 0; i < 4; ++i) t4[i] = b1 ? t8[2 * i + 1] : t8[2 * i];
#pragma unroll
    for (int i = 0; i < 2; ++i) t2[i] = b2 ? t4[2 * i + 1] : t4[2 * i];
    return b3 ? t2[1] : t2[0];
}

__device__ __forceinline__ void add_bias16(float* v, const float* b, int c)
{
#pragma unroll
    for (int j = 0; j < 16; j += 4) {
        const float4 bb = ld_bias4(b, c + j);
        v[j] += bb.x;
        v[j + 1] += bb.y;
        v[j + 2] += bb.z;
        v[j + 3] += bb.w;
    }
}

__device__ __forceinline__ bool train_epilogue(const DecArgs& a, const float* bias, EpiCtx& e, int ntiles,
                                               float& acc_ce, float& acc_u, float& acc_l1)
{
    constexpr float kL2E = 1.4426950408889634f;
    const int row = e.row, h = e.h;
    const float *b1s = bias, *b2s = bias + kH1, *b3s = bias + kH1 + kH2;
    const uint32_t tl = e.tw + e.lanef;
    const int nu = a.ncb / 16, per = (nu + 1) / 2;
    const int c0 = min(nu, h * per) * 16, c1 = min(nu, (h + 1) * per) * 16;   // this half's logit columns
    float v[16];
    // this row's inputs of the slot's next tile, loaded one tile ahead so that
    // their latency is not on the path from one tile's first MMA to the next:
    // half 0 the feature, half 1 (with the L1 term) the image and its target
    float pf[8], pu = 0.f;
    int pt = -1;
    auto fetch = [&](int tile_n) {
        const int pxn = tile_n * 128 + row;
        const bool vn = tile_n < ntiles && pxn < a.P;
        if (h == 0) {
#pragma unroll
            for (int c = 0; c < 8; ++c) pf[c] = vn ? a.feat[(size_t)c * a.P + pxn] : 0.f;
        } else if (a.img) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                pf[c] = vn ? a.img[(size_t)c * a.P + pxn] : 0.f;
                pf[3 + c] = vn ? a.img_t[(size_t)c * a.P + pxn] : 0.f;
            }
        }
        pu = vn ? a.unc[pxn] : 0.f;
        pt = vn ? a.target[pxn] : -1;
    };
    fetch(blockIdx.x + e.s * gridDim.x);
    for (int it = 0;; ++it) {
        const int tile = blockIdx.x + (2 * it + e.s) * gridDim.x;
        if (tile >= ntiles) break;
        const int px = tile * 128 + row;
        const bool valid = px < a.P;
        const uint32_t sb = opaque(e.sb);
        const uint32_t X1 = sb + kSX1, H1 = sb + kSH1, H2 = sb + kSH2, D = sb + kSD;
        // X1 = [feat | 1 | 0]: the ones column gives db1
        if (h == 0) {
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] = pf[c];
            sts_bf16x8(X1 + sbuf_off(row, 0, 16), v);
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) v[c] = c == 0 ? 1.f : 0.f;
            sts_bf16x8(X1 + sbuf_off(row, 8, 16), v);
            if (a.img && valid) {
                // the RGB L1 term of this pixel (the same operations as le_rgb_l1)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float r = pf[c] - pf[3 + c];
                    acc_l1 += fabsf(r);
                    a.d_img[(size_t)c * a.P + px] = r > 0.f ? a.inv_l1 : (r < 0.f ? -a.inv_l1 : 0.f);
                }
            }
        }
        const float u = pu;
        const int t = pt;
        fetch(tile + 2 * (int)gridDim.x);
        epi_signal(e);
        if (!epi_wait(e)) return false;
        // E1: h1 columns [32h, 32h + 32), bits of the ReLU mask in m1
        uint32_t m1 = 0;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            tmem_ld16(tl + 32 * h + 16 * k, v);
            m1 |= bias_relu16(v, b1s, 32 * h + 16 * k) << (16 * k);
            store16(H1, kH1, row, 32 * h + 16 * k, v);
        }
        epi_signal(e);
        if (!epi_wait(e)) return false;
        // E2: h2 columns [64h, 64h + 64), mask bits in m2a (first 32) and m2b
        uint32_t m2a = 0, m2b = 0;
#pragma unroll 1
        for (int k = 0; k < 4; ++k) {
            tmem_ld16(tl + 64 * h + 16 * k, v);
            const uint32_t mk = bias_relu16(v, b2s, 64 * h + 16 * k);
            if (k < 2) m2a |= mk << (16 * k);
            else m2b |= mk << (16 * (k - 2));
            store16(H2, 128, row, 64 * h + 16 * k, v);
        }
        epi_signal(e);
        if (!epi_wait(e)) return false;
        // E3: softmax over this half's logit columns [c0, c1).  Pass 1: max (and
        // the target's logit); pass 2: e = exp(z - max), their sum, e parked in
        // the free TMEM columns; exchange with the other half; pass 3: dz.
        const int jt = t - c0;
        const bool own_t = jt >= 0 && t < c1;
        float mh = -INFINITY, zt_h = 0.f;
#pragma unroll 1
        for (int uu = 0; uu < 4; ++uu)
            if (c0 + 16 * uu < c1) {
                tmem_ld16(tl + c0 + 16 * uu, v);
                add_bias16(v, b3s, c0 + 16 * uu);
#pragma unroll
                for (int j = 0; j < 16; ++j) mh = fmaxf(mh, v[j]);
                if (own_t && (jt >> 4) == uu) zt_h = select16(v, jt & 15);
            }
        const float mhl = mh * kL2E;
        float sh = 0.f;
#pragma unroll 1
        for (int uu = 0; uu < 4; ++uu)
            if (c0 + 16 * uu < c1) {
                tmem_ld16(tl + c0 + 16 * uu, v);
                add_bias16(v, b3s, c0 + 16 * uu);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    v[j] = ex2_approx(fmaf(v[j], kL2E, -mhl));
                    sh += v[j];
                }
                tmem_st16(tl + c0 + 16 * uu, v);
            }
        tmem_wait_st();
        // the halves exchange (max, sum, target logit) through D's columns [0, 16),
        // which pass 3 then overwrites with dz: no stale FP32 bits stay in D to
        // reach an MMA (as bf16 they can be Inf or NaN)
        float4 o;
        asm volatile("st.shared.v4.f32 [%0], {%1,%2,%3,%4};" ::"r"(D + xch_off(h * 128 + row)), "f"(mh), "f"(sh),
                     "f"(zt_h), "f"(0.f)
                     : "memory");
        asm volatile("bar.sync %0, 256;" ::"r"(e.bar_id) : "memory");
        asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
                     : "=f"(o.x), "=f"(o.y), "=f"(o.z), "=f"(o.w)
                     : "r"(D + xch_off((1 - h) * 128 + row))
                     : "memory");
        asm volatile("bar.sync %0, 256;" ::"r"(e.bar_id) : "memory");
        const float m = fmaxf(mh, o.x);
        const float ssum = (c0 < c1 ? sh * ex2_approx((mh - m) * kL2E) : 0.f) +
                           (o.y > 0.f ? o.y * ex2_approx((o.x - m) * kL2E) : 0.f);
        const float lse = m + __logf(ssum);
        const float zt = own_t ? zt_h : o.z;
        const float ce = lse - zt;
        const float w = valid ? a.lambda_ce * (1.f - u) : 0.f;
        if (valid && h == 0) {
            a.d_unc[px] = (a.lambda_u - a.lambda_ce * ce) * a.invP;
            acc_ce += ce * (1.f - u);
            acc_u += u;
        }
        // dz * P (1/P is applied when the gradients are written)
        const float scale = c0 < c1 ? w * ex2_approx((mh - m) * kL2E) / ssum : 0.f;
#pragma unroll 1
        for (int uu = 0; uu < 4; ++uu)
            if (c0 + 16 * uu < c1) {
                tmem_ld16(tl + c0 + 16 * uu, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] *= scale;
                store16(D, 128, row, c0 + 16 * uu, v);
            }
        if (own_t && valid) {
            const float et = ex2_approx(fmaf(zt_h, kL2E, -mhl));
            const __nv_bfloat16 bv = __float2bfloat16_rn(et * scale - w);
            asm volatile("st.shared.b16 [%0], %1;" ::"r"(D + sbuf_off(row, t, 128)),
                         "h"(*reinterpret_cast<const unsigned short*>(&bv))
                         : "memory");
        }
        epi_signal(e);
        if (!epi_wait(e)) return false;
        // E4: dh2 = (dz W3) * [h2 > 0] into H2's buffer
#pragma unroll 1
        for (int k = 0; k < 4; ++k) {
            tmem_ld16(tl + 64 * h + 16 * k, v);
            mask16(v, (k < 2 ? m2a : m2b) >> (16 * (k & 1)));
            store16(H2, 128, row, 64 * h + 16 * k, v);
        }
        epi_signal(e);
        if (!epi_wait(e)) return false;
        // E5: dh1 = (dh2 W2) * [h1 > 0] into D
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            tmem_ld16(tl + 32 * h + 16 * k, v);
            mask16(v, m1 >> (16 * k));
            store16(D, 128, row, 32 * h + 16 * k, v);
        }
        epi_signal(e);
        if (!epi_wait(e)) return false;
        // E6: dx = dh1 W1 -> d_feat
        if (h == 0) {
            tmem_ld16(tl, v);
            if (valid)
#pragma unroll
                for (int c = 0; c < kD; ++c) a.d_feat[(size_t)c * a.P + px] = v[c] * a.invP;
        }
    }
    return true;
}

__global__ void __launch_bounds__(kTrainThreads, 1) dec_train_kernel(DecArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    Front f;
    unsigned char* p = load_weights(sm, a, f);
    const SBuf E{p, kEC};
    p += sbuf_bytes(128, kEC);
    unsigned char* slots = p;
    const uint32_t slots_a = smem_u32(slots);
    p += 2 * train_slot_bytes();
    uint64_t* ready = reinterpret_cast<uint64_t*>(p);
    uint64_t* done = ready + 2;
    uint64_t* fin = ready + 4;
    uint32_t* slot_addr = reinterpret_cast<uint32_t*>(ready + 5);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the slots start zeroed (padding columns feed MMA rows that are never read,
    // and must hold finite values); E has ones in columns 8 and 17
    for (size_t i = threadIdx.x; i < 2 * train_slot_bytes() / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(slots)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = threadIdx.x; i < 128 * (kEC / 8); i += blockDim.x) {
        const int r = i / (kEC / 8), cb = i % (kEC / 8);
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (cb == 1) v[0] = 1.f;
        if (cb == 2) v[1] = 1.f;
        sbuf_store8(E, r, 8 * cb, v);
    }
    if (threadIdx.x == 0) {
        mbar_init(ready, 256);
        mbar_init(ready + 1, 256);
        mbar_init(done, 1);
        mbar_init(done + 1, 1);
        mbar_init(fin, 1);
    }
    if (warp == 0) tmem_alloc(slot_addr, 512);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tb = *reinterpret_cast<volatile uint32_t*>(slot_addr);
    const int ntiles = (a.P + 127) / 128;
    bool ok = true;
    float acc_ce = 0.f, acc_u = 0.f, acc_l1 = 0.f;
    if (warp == 16) {
        if (lane == 0) {
            ok = train_mma_loop(a.ncb, f, smem_u32(E.p), slots_a, ready, done, tb, ntiles);
            if (ok) {
                commit(fin);
                ok = mbar_wait(fin, 0);
            }
        }
    } else {
        EpiCtx e;
        e.s = warp >> 3;
        e.h = (warp >> 2) & 1;
        e.row = threadIdx.x & 127;
        e.sb = slots_a + kSlotBytes * e.s;
        e.ready = ready + e.s;
        e.done = done + e.s;
        e.tw = tb + 128u * e.s;
        e.lanef = (uint32_t)(32 * (warp & 3)) << 16;
        e.ph = 0;
        e.bar_id = 1 + e.s;
        ok = train_epilogue(a, f.b1s, e, ntiles, acc_ce, acc_u, acc_l1);
    }
    fence_before();
    const bool bad = __syncthreads_or(!ok);
    fence_after();
    if (bad) {
        if (threadIdx.x == 0) atomicExch(&g_tc_error, 1);
    } else if (warp < 16) {
        // flush the weight-gradient accumulators: TMEM lane = this thread's row
        const int row = threadIdx.x & 127, wg = warp >> 2;
        const uint32_t lanef = (uint32_t)(32 * (warp & 3)) << 16;
        float v[16];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            tmem_ld16(tb + kTW3 + lanef + 32 * wg + 16 * k, v);
            if (row < a.ncb)
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    atomicAdd(a.dW3 + (size_t)row * kH2 + 32 * wg + 16 * k + j, v[j] * a.invP);
        }
        tmem_ld16(tb + kTW2 + lanef + 16 * wg, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) atomicAdd(a.dW2 + (size_t)row * kH1 + 16 * wg + j, v[j] * a.invP);
        if (wg == 0) {
            tmem_ld16(tb + kTP + lanef, v);
            atomicAdd(a.db2 + row, v[0] * a.invP);
            if (row < a.ncb) atomicAdd(a.db3 + row, v[8] * a.invP);
        } else if (wg == 1) {
            tmem_ld16(tb + kTQ + lanef, v);
            if (row < kH1) {
#pragma unroll
                for (int j = 0; j < kD; ++j) atomicAdd(a.dW1 + (size_t)row * kD + j, v[j] * a.invP);
                atomicAdd(a.db1 + row, v[kD] * a.invP);
            }
        }
    }
    if (warp < 16) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc_ce += __shfl_xor_sync(0xffffffffu, acc_ce, o);
            acc_u += __shfl_xor_sync(0xffffffffu, acc_u, o);
            acc_l1 += __shfl_xor_sync(0xffffffffu, acc_l1, o);
        }
        if (lane == 0 && ((warp >> 2) & 1) == 0) {
            atomicAdd(a.loss, acc_ce * a.invP);
            atomicAdd(a.loss + 1, acc_u * a.invP);
        }
        if (lane == 0 && ((warp >> 2) & 1) == 1 && a.loss_l1) atomicAdd(a.loss_l1, acc_l1 * a.inv_l1);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(tb, 512);
}

// ---------------------------------------------------------------------------
// Query: decode, softmax (unnormalised), relevancy.  Four warpgroups per CTA serve the same
// 128 rows and split every epilogue by columns; TMEM: logits in [0, ncb)
// (later the 16 text/negative projections in [0, 16) and the four parts'
// partial p^T G p in columns 16-19), p^T G in [256, 256 + ncb).  The
// activations X1/H1/H2, the parts' softmax exchange and the BF16 softmax P
// share one region (each is written after the last reader of the previous
// one has finished).
constexpr uint32_t kTG = 256;
constexpr int kQueryParts = 4;

__host__ constexpr size_t query_smem(int ncb)
{
    return weights_bytes(ncb) + sbuf_bytes(16, ncb) +
           (sbuf_bytes(128, ncb) > kFwdWgBytes ? sbuf_bytes(128, ncb) : kFwdWgBytes) + 2 * sbuf_bytes(ncb, 64) + 128;
}

__global__ void __launch_bounds__(128 * kQueryParts, 1) query_fused_kernel(DecArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    Front f;
    unsigned char* p = load_weights(sm, a, f);
    const SBuf Aqs{p, a.ncb};
    p += sbuf_bytes(16, a.ncb);
    f.X1 = SBuf{p, 16};
    f.H1 = SBuf{p + sbuf_bytes(128, 16), 64};
    f.H2 = SBuf{p + sbuf_bytes(128, 16) + sbuf_bytes(128, 64), 128};
    const SBuf Ps{p, a.ncb};
    f.xch = reinterpret_cast<float4*>(p);
    p += sbuf_bytes(128, a.ncb) > kFwdWgBytes ? sbuf_bytes(128, a.ncb) : kFwdWgBytes;
    // G in 64-column chunks: chunks 0 and 1 stay in their own slots for the whole
    // kernel; chunks 2 and 3 (n_cb > 128) go into W3's shared memory, which
    // holds exactly two chunks and is idle from the end of the third layer's
    // MMAs to the next tile's: they are copied in while the softmax runs, and
    // W3 is copied back (from its global image) while the relevancy and the
    // next tile's first two layers run, so no copy is on the tile's path.
    const uint32_t chunk_bytes = sbuf_bytes(a.ncb, 64);
    unsigned char* const g_own = p;
    auto g_chunk = [&](int kc) {
        return SBuf{kc < 2 ? g_own + kc * chunk_bytes : f.W3s.p + (kc - 2) * chunk_bytes, 64};
    };
    p += 2 * chunk_bytes;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(p);     // [0] MMA, [1] chunks 0-1, [2] chunks 2-3, [4] W3
    uint32_t* slot = reinterpret_cast<uint32_t*>(p + 24);
    const int tid = threadIdx.x;
    sbuf_fill(Aqs, 16, a.Aq, a.ncb, 16, a.ncb);
    f.mbar = mbar;
    f.phase = 0;
    f.tid = tid & 127;
    f.bar_id = 0;
    f.nthreads = blockDim.x;
    f.half = tid >> 7;
    f.nhalf = kQueryParts;
    f.w3bar = mbar + 4;
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) mbar_init(mbar + i, 1);
        mbar_init(mbar + 4, 1);
    }
    if (tid < 32) tmem_alloc(slot, 512);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(slot);
    f.tw = tbase;
    f.lane = (uint32_t)(32 * ((tid >> 5) & 3)) << 16;
    const int row = f.tid;
    int c0, c1;
    my_cols(f, a.ncb, c0, c1);                  // this part's class columns
    const int nch = a.ncb / 64;                 // G chunks (64 K-columns each)
    const int nlow = nch < 2 ? nch : 2, nup = nch - nlow;
    // loads in flight (thread 0 only): chunks 0-1 (once), chunks 2-3 (per tile)
    bool low_pending = false, up_pending = false;
    uint32_t up_phase = 0u;
    const int ntiles = (a.P + 127) / 128;
    bool ok = true;
    if (tid == 0 && blockIdx.x < ntiles) {
        mbar_expect_tx(mbar + 1, nlow * chunk_bytes);
        bulk_g2s(g_own, a.G_img, nlow * chunk_bytes, mbar + 1);
        low_pending = true;
    }
    float xf[8];                                // this tile's R_s, loaded a tile ahead (part 0)
    if (f.half == 0) load_feat(a, blockIdx.x * 128 + row, blockIdx.x * 128 + row < a.P, xf);
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int px = tile * 128 + row;
        const bool valid = px < a.P;
        if (!mlp_forward_x(f, a, xf)) break;
        // the third layer's MMAs have read W3: chunks 2-3 of G take its place
        if (tid == 0 && nup > 0) {
            mbar_expect_tx(mbar + 2, nup * chunk_bytes);
            bulk_g2s(f.W3s.p, a.G_img + 2 * (size_t)chunk_bytes, nup * chunk_bytes, mbar + 2);
            up_pending = true;
        }
        if (f.half == 0) {
            const int nx = px + 128 * (int)gridDim.x;
            load_feat(a, nx, tile + (int)gridDim.x < ntiles && nx < a.P, xf);
        }
        // e = exp(z - max z) in BF16.  The relevancy phi.q / |phi| with
        // phi = sum_c p_c s_c does not depend on the scale of p, so the
        // softmax normaliser 1 / sum e is never needed.
        float v[16], mh = -INFINITY;
        for (int c = c0; c < c1; c += 16) {
            tmem_ld16(f.tw + f.lane + c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) mh = fmaxf(mh, v[j] + f.b3s[c + j]);
        }
        f.xch[f.half * 128 + row].x = mh;
        wg_sync(f);
        float m = -INFINITY;
#pragma unroll
        for (int h = 0; h < kQueryParts; ++h) m = fmaxf(m, f.xch[h * 128 + row].x);
        wg_sync(f);
        const float ml = m * 1.4426950408889634f;
        for (int c = c0; c < c1; c += 16) {
            tmem_ld16(f.tw + f.lane + c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = ex2_approx(fmaf(v[j] + f.b3s[c + j], 1.4426950408889634f, -ml));
            sbuf_store8(Ps, row, c, v);
            sbuf_store8(Ps, row, c + 8, v + 8);
        }
        wg_publish(f);
        // p . (S_c [q; n]) into [0, 16), p^T G into [256, 256 + ncb), all chunks in one round
        bool tmo = false;
        if (tid == 0) {
            for (int s = 0; s < a.ncb / 16; ++s)
                mma(tbase, kdesc(Ps, 0, 16 * s), kdesc(Aqs, 0, 16 * s), idesc_bf16(16, false, false), s > 0);
            if (low_pending) {
                if (!mbar_wait(mbar + 1, 0u)) tmo = true;
                low_pending = false;
            }
            for (int kc = 0; kc < nch; ++kc) {
                if (kc == 2) {
                    if (!mbar_wait(mbar + 2, up_phase)) tmo = true;
                    up_phase ^= 1u;
                    up_pending = false;
                }
                for (int k = 0; k < 4; ++k)
                    mma(tbase + kTG, kdesc(Ps, 0, 64 * kc + 16 * k), kdesc(g_chunk(kc), 0, 16 * k),
                        idesc_bf16(a.ncb, false, false), kc > 0 || k > 0);
            }
            commit(f.mbar);
        }
        if (!wg_wait(f) || bar_any(0, blockDim.x, tmo)) {
            if (tid == 0) atomicExch(&g_tc_error, 1);
            break;
        }
        // the G MMAs are done with W3's shared memory: W3 goes back for the next tile
        if (tid == 0 && nup > 0 && tile + (int)gridDim.x < ntiles) {
            mbar_expect_tx(f.w3bar, sbuf_bytes(a.ncb, 128));
            bulk_g2s(f.W3s.p, a.W3_img, sbuf_bytes(a.ncb, 128), f.w3bar);
            f.w3pending = true;
        }
        // relevancy: each part sums e^T G e over its columns into TMEM column 16 + part
        float ptgp = 0.f, pp[16];
        for (int c = c0; c < c1; c += 16) {
            tmem_ld16(tbase + kTG + f.lane + c, v);
            sbuf_load8(Ps, row, c, pp);
            sbuf_load8(Ps, row, c + 8, pp + 8);
#pragma unroll
            for (int j = 0; j < 16; ++j) ptgp = fmaf(pp[j], v[j], ptgp);
        }
        tmem_st1(tbase + f.lane + 16 + f.half, ptgp);
        tmem_wait_st();
        fence_before();
        __syncthreads();
        fence_after();
        if (f.half == 0) {
            tmem_ld16(tbase + f.lane, v);        // the 16 projections and the parts' partial sums
            float tot = 0.f, w[16];
            tmem_ld16(tbase + f.lane + 16, w);
#pragma unroll
            for (int h = 0; h < kQueryParts; ++h) tot += w[h];
            const float inv = rsqrtf(fmaxf(tot, 1e-30f));
            // unrolled with constant indices: v stays in registers (a runtime
            // index would put it, and every TMEM load into it, in local memory)
            float smax = -INFINITY;
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (j >= a.Q && j < a.Q + a.n_neg) smax = fmaxf(smax, v[j] * inv);
            if (valid)
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (j < a.Q) a.rel[(size_t)j * a.P + px] = 1.f / (1.f + __expf(smax - v[j] * inv));
        }
        fence_before();
        __syncthreads();
    }
    // drain copies still in flight (only after an early exit) before the shared memory goes away
    if (tid == 0) {
        if (low_pending) mbar_wait(mbar + 1, 0u);
        if (up_pending) mbar_wait(mbar + 2, up_phase);
        if (f.w3pending) mbar_wait(f.w3bar, f.w3phase);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (tid < 32) tmem_dealloc(tbase, 512);
}

// ---------------------------------------------------------------------------
// Language feature map export F = M_infer S (supp. Sec. "Inference"): per
// pixel the decoder's softmax p over the n_cb codes times the codebook, in
// BF16.  Four warpgroups serve the same 128 rows as in the query kernel; e =
// exp(z - max z) is stored in BF16 and each output row is scaled by 1/sum e.
// The codebook streams through shared memory in 64-dim chunks ([n_cb x 64]
// canonical images, two slots, 1-D bulk copies); per chunk one MMA (M = 128
// pixels, N = 64 dims, K = n_cb) reads the chunk MN-major into one of two
// 64-column TMEM accumulators.  Each warpgroup converts 16 columns of each
// into a 128-byte-swizzled staging area, from which two TMA tensor stores per
// round (128 pixels x 64 dims each) write the output in whole lines; a warp
// storing its rows directly would scatter 16-byte pieces over 32 rows.
constexpr uint32_t kTF = 256;      // TMEM columns of the two chunk accumulators

// Shared memory of the export kernel without the output staging, the staging
// (one round's two 128 x 64 BF16 boxes, 128-byte swizzled for the TMA store),
// and whether the staging must borrow W3's shared memory (then W3 is reloaded
// from its global image after every tile; it is idle during the codebook loop).
// The layout starts at a 1024-byte boundary (the swizzled staging and W3s, at
// offset 18 KB, need it), hence the first 1024.
__host__ constexpr size_t export_smem_core(int ncb)
{
    return 1024 + weights_bytes(ncb) + (sbuf_bytes(128, ncb) > kFwdWgBytes ? sbuf_bytes(128, ncb) : kFwdWgBytes) +
           2 * sbuf_bytes(ncb, 64) + kQueryParts * 128 * 4 + 128;
}
constexpr uint32_t kExportBox = sbuf_bytes(128, 64);
constexpr size_t kMaxDynSmem = 227 * 1024;
__host__ constexpr bool export_stage_in_w3(int ncb) { return export_smem_core(ncb) + 1024 + 2 * kExportBox > kMaxDynSmem; }
__host__ constexpr size_t export_smem(int ncb)
{
    return export_smem_core(ncb) + (export_stage_in_w3(ncb) ? 0 : 1024 + 2 * kExportBox);
}

__global__ void __launch_bounds__(128 * kQueryParts, 1) export_fused_kernel(const __grid_constant__ CUtensorMap tmap_out,
                                                                          DecArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    Front f;
    unsigned char* p = load_weights(
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sm) + 1023) & ~uintptr_t(1023)), a, f);
    f.X1 = SBuf{p, 16};
    f.H1 = SBuf{p + sbuf_bytes(128, 16), 64};
    f.H2 = SBuf{p + sbuf_bytes(128, 16) + sbuf_bytes(128, 64), 128};
    const SBuf Ps{p, a.ncb};
    f.xch = reinterpret_cast<float4*>(p);
    p += sbuf_bytes(128, a.ncb) > kFwdWgBytes ? sbuf_bytes(128, a.ncb) : kFwdWgBytes;
    const uint32_t chunk_bytes = sbuf_bytes(a.ncb, 64);
    const SBuf Gs[2] = {SBuf{p, 64}, SBuf{p + chunk_bytes, 64}};
    p += 2 * chunk_bytes;
    float* sums = reinterpret_cast<float*>(p);          // [parts][128] partial sums of e
    p += kQueryParts * 128 * 4;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(p);     // [0] MMA, [1], [2] codebook slots, [4] W3 reload
    uint32_t* slot = reinterpret_cast<uint32_t*>(p + 24);
    p += 128;
    unsigned char* stg = a.w3_reload ? f.W3s.p
                                     : reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) &
                                                                        ~uintptr_t(1023));
    const int tid = threadIdx.x;
    f.mbar = mbar;
    f.phase = 0;
    f.tid = tid & 127;
    f.bar_id = 0;
    f.nthreads = blockDim.x;
    f.half = tid >> 7;
    f.nhalf = kQueryParts;
    f.w3bar = mbar + 4;
    if (tid == 0) {
        for (int i = 0; i < 3; ++i) mbar_init(mbar + i, 1);
        mbar_init(mbar + 4, 1);
    }
    if (tid < 32) tmem_alloc(slot, 512);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(slot);
    f.tw = tbase;
    f.lane = (uint32_t)(32 * ((tid >> 5) & 3)) << 16;
    const int row = f.tid;
    int c0, c1;
    my_cols(f, a.ncb, c0, c1);
    const int nch = a.dd / 64;
    uint32_t gphase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    auto load_chunk = [&](int kc, int s) {
        mbar_expect_tx(mbar + 1 + s, chunk_bytes);
        bulk_g2s(Gs[s].p, a.G_img + (size_t)kc * chunk_bytes, chunk_bytes, mbar + 1 + s);
        pending[s] = true;
    };
    const int ntiles = (a.P + 127) / 128;
    bool ok = true;
    if (tid == 0 && blockIdx.x < ntiles)
        for (int s = 0; s < 2 && s < nch; ++s) load_chunk(s, s);
    float xf[8];                                // this tile's R_s, loaded a tile ahead (part 0)
    if (f.half == 0) load_feat(a, blockIdx.x * 128 + row, blockIdx.x * 128 + row < a.P, xf);
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int px = tile * 128 + row;
        const bool valid = px < a.P;
        if (!mlp_forward_x(f, a, xf)) break;
        if (f.half == 0) {
            const int nx = px + 128 * (int)gridDim.x;
            load_feat(a, nx, tile + (int)gridDim.x < ntiles && nx < a.P, xf);
        }
        float v[16], mh = -INFINITY;
        for (int c = c0; c < c1; c += 16) {
            tmem_ld16(f.tw + f.lane + c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) mh = fmaxf(mh, v[j] + f.b3s[c + j]);
        }
        f.xch[f.half * 128 + row].x = mh;
        wg_sync(f);
        float m = -INFINITY;
#pragma unroll
        for (int h = 0; h < kQueryParts; ++h) m = fmaxf(m, f.xch[h * 128 + row].x);
        wg_sync(f);
        const float ml = m * 1.4426950408889634f;
        float se = 0.f;
        for (int c = c0; c < c1; c += 16) {
            tmem_ld16(f.tw + f.lane + c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                v[j] = ex2_approx(fmaf(v[j] + f.b3s[c + j], 1.4426950408889634f, -ml));
                se += v[j];
            }
            sbuf_store8(Ps, row, c, v);
            sbuf_store8(Ps, row, c + 8, v + 8);
        }
        sums[f.half * 128 + row] = se;
        wg_publish(f);
        float tot = 0.f;
#pragma unroll
        for (int h = 0; h < kQueryParts; ++h) tot += sums[h * 128 + row];
        const float inv = valid ? 1.0f / tot : 0.f;
        bool tmo = false;
        for (int kc0 = 0; kc0 < nch; kc0 += 2) {
            if (tid == 0) {
                for (int s = 0; s < 2 && kc0 + s < nch; ++s) {
                    if (!mbar_wait(mbar + 1 + s, gphase[s])) tmo = true;
                    gphase[s] ^= 1u;
                    pending[s] = false;
                    const uint64_t gm = mndesc(Gs[s], 0, 0);
                    for (int k = 0; k < a.ncb / 16; ++k)
                        mma(tbase + kTF + 64 * s, kdesc(Ps, 0, 16 * k), gm + 128 * k, idesc_bf16(64, false, true),
                            k > 0);
                }
                commit(f.mbar);
                // the staging area is rewritten below: the previous round's stores must have read it
                bulk_wait_read_all();
            }
            if (!wg_wait(f) || bar_any(0, blockDim.x, tmo)) {
                if (tid == 0) atomicExch(&g_tc_error, 1);
                ok = false;
                break;
            }
            // refill the slots: the next chunk pair of this tile, or the first pair of the next tile
            if (tid == 0) {
                const bool more = kc0 + 2 < nch;
                const bool next_tile = tile + (int)gridDim.x < ntiles;
                for (int s = 0; s < 2; ++s) {
                    const int kc = more ? kc0 + 2 + s : s;
                    if ((more && kc < nch) || (!more && next_tile && kc < nch)) load_chunk(kc, s);
                }
            }
            // this warpgroup's 16 columns of each chunk, scaled by 1 / sum e, as BF16 into the
            // staging boxes (row-major 128-byte rows, 16-byte unit u of row r at u ^ (r & 7))
            for (int s = 0; s < 2 && kc0 + s < nch; ++s) {
                tmem_ld16(tbase + kTF + 64 * s + 16 * f.half + f.lane, v);
                __nv_bfloat162 h[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(v[2 * j] * inv, v[2 * j + 1] * inv);
                unsigned char* dst = stg + s * kExportBox + row * 128;
                const int u = 2 * f.half;
                *reinterpret_cast<uint4*>(dst + ((u ^ (row & 7)) << 4)) = *reinterpret_cast<uint4*>(h);
                *reinterpret_cast<uint4*>(dst + (((u + 1) ^ (row & 7)) << 4)) = *reinterpret_cast<uint4*>(h + 4);
            }
            fence_proxy_async();
            fence_before();
            __syncthreads();
            fence_after();
            if (tid == 0) {
                for (int s = 0; s < 2 && kc0 + s < nch; ++s)
                    tma_store_2d(&tmap_out, 64 * (kc0 + s), tile * 128, stg + s * kExportBox);
                bulk_commit();
                // after the tile's last round, W3 goes back into the staging area for the next tile
                if (a.w3_reload && kc0 + 2 >= nch && tile + (int)gridDim.x < ntiles) {
                    bulk_wait_read_all();
                    mbar_expect_tx(f.w3bar, sbuf_bytes(a.ncb, 128));
                    bulk_g2s(f.W3s.p, a.W3_img, sbuf_bytes(a.ncb, 128), f.w3bar);
                    f.w3pending = true;
                }
            }
        }
    }
    // drain copies still in flight before the shared memory goes away
    if (tid == 0) {
        for (int s = 0; s < 2; ++s)
            if (pending[s]) mbar_wait(mbar + 1 + s, gphase[s]);
        if (f.w3pending) mbar_wait(f.w3bar, f.w3phase);
        bulk_wait_all();
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (tid < 32) tmem_dealloc(tbase, 512);
}

// W3 [ncb x 128] (fp32) -> its BF16 shared-memory image (the layout load_weights writes).
__global__ void w3_image_kernel(const float* __restrict__ W3, int ncb, unsigned char* __restrict__ img)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncb * (kH2 / 8); i += gridDim.x * blockDim.x) {
        const int r = i / (kH2 / 8), c0 = (i % (kH2 / 8)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = W3[(size_t)r * kH2 + c0 + j];
        sbuf_store8(SBuf{img, kH2}, r, c0, v);
    }
}

// Codebook S [ncb x dd] (fp32) -> chunked canonical bf16 image: chunk kc holds
// dims [64 kc, 64 kc + 64) of every code, as an [ncb x 64] canonical buffer.
__global__ void codebook_chunks_kernel(const float* __restrict__ S, int ncb, int dd, unsigned char* __restrict__ img)
{
    const int n8 = ncb * (dd / 8);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += gridDim.x * blockDim.x) {
        const int r = i / (dd / 8), c0 = (i % (dd / 8)) * 8;
        const int kc = c0 / 64, cc = c0 % 64;
        __nv_bfloat162 h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            h[j] = __floats2bfloat162_rn(S[(size_t)r * dd + c0 + 2 * j], S[(size_t)r * dd + c0 + 2 * j + 1]);
        unsigned char* dst = img + (size_t)kc * ncb * 64 * 2 + ((r >> 3) * 8 * 128 + (cc >> 3) * 128 + (r & 7) * 16);
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<uint4*>(h);
    }
}

// Query constants in one launch, 16 x 16 outputs per block, k ascending with
// FMAs (the order of a plain dot product):
//   block rows y < ncb/16:  G = S_c S_c^T, written straight into its chunked
//                           canonical BF16 image: chunk kc holds columns
//                           [64 kc, 64 kc + 64) of every row as an [ncb x 64]
//                           canonical buffer;
//   block row y = ncb/16:   Aq[r][j] = [text; negs]_r . S_c[j] (rows r >= Q + n_neg zero).
__global__ void __launch_bounds__(256) query_prep_kernel(const float* __restrict__ S, int ncb, int dd, int d_clip,
                                                         const float* __restrict__ text, int Q,
                                                         const float* __restrict__ negs, int n_neg,
                                                         unsigned char* __restrict__ img, float* __restrict__ Aq)
{
    __shared__ float xs[16][33], ys[16][33];
    const int j0 = blockIdx.x * 16, i0 = blockIdx.y * 16;
    const bool gram = i0 < ncb;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc = 0.f;
    for (int k0 = 0; k0 < d_clip; k0 += 32) {
        for (int l = threadIdx.x; l < 16 * 32; l += 256) {
            const int r = l >> 5, c = l & 31, k = k0 + c;
            float xv = 0.f;
            if (k < d_clip) {
                if (gram) xv = S[(size_t)(i0 + r) * dd + k];
                else if (r < Q) xv = text[(size_t)r * d_clip + k];
                else if (r < Q + n_neg) xv = negs[(size_t)(r - Q) * d_clip + k];
            }
            xs[r][c] = xv;
            ys[r][c] = k < d_clip ? S[(size_t)(j0 + r) * dd + k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 32; ++c) acc = fmaf(xs[ty][c], ys[tx][c], acc);
        __syncthreads();
    }
    const int r = i0 + ty, c = j0 + tx;
    if (gram) {
        const int kc = c >> 6, cc = c & 63;
        unsigned char* dst = img + (size_t)kc * ncb * 64 * 2 + ((r >> 3) * 8 * 128 + (cc >> 3) * 128 + (r & 7) * 16) +
                             (cc & 7) * 2;
        *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(acc);
    } else {
        Aq[(size_t)ty * ncb + c] = acc;
    }
}

// Self-test of the bounded-wait path: waits on an mbarrier that nothing ever
// arrives at, gives up after the usual limit and records the timeout.
__global__ void selftest_wait_kernel()
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(&bar, 0u)) atomicExch(&g_tc_error, 1);
}

// Up to eight FP32 arrays set to zero in one launch (block i clears array i).
struct ZeroList {
    float* p[8];
    int n[8];
};
__global__ void __launch_bounds__(256) zero_list_kernel(ZeroList z)
{
    float* p = z.p[blockIdx.x];
    const int n = z.n[blockIdx.x];
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0.f;
}

// SM count of the calling thread's current device, read on every launch (a
// cheap attribute query), so a process driving parts of different sizes gets
// each one's own persistent grid.
int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        n = 1;
    return n;
}

template <class K>
le_status set_smem(K kernel, size_t bytes)
{
    LE_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return LE_OK;
}

}  // namespace

le_status check_fused_decoder(const le_decoder* d, bool train)
{
    if (d->d_in != kD || d->h1 != kH1 || d->h2 != kH2 || d->n_cb % 16 != 0 || d->n_cb < 16 || d->n_cb > 256 ||
        (train && d->n_cb > 128)) {
        set_error("fused path supports d_in=8, h1=64, h2=128, n_cb multiple of 16 in [16, %d]; got %d-%d-%d-%d",
                  train ? 128 : 256, d->d_in, d->h1, d->h2, d->n_cb);
        return LE_ERR_UNSUPPORTED;
    }
    return LE_OK;
}

size_t decode_fused_workspace(int32_t, const le_decoder*) { return 0; }

le_status decode_fused(int32_t P, const float* feat, const float* unc, const le_decoder* d, const int32_t* target,
                       float lambda_ce, float lambda_u, float* loss, float* d_feat, float* d_unc,
                       const le_decoder_grads* dg, int32_t* argmax, float* prob, void*, size_t, cudaStream_t s,
                       const float* img, const float* img_t, float* loss_l1, float* d_img)
{
    DecArgs a{};
    a.img = img;
    a.img_t = img_t;
    a.loss_l1 = loss_l1;
    a.d_img = d_img;
    a.inv_l1 = 1.0f / (float)(3 * (int64_t)P);
    a.P = P;
    a.ncb = d->n_cb;
    a.feat = feat;
    a.unc = unc;
    a.target = target;
    a.W1 = d->W1; a.b1 = d->b1; a.W2 = d->W2; a.b2 = d->b2; a.W3 = d->W3; a.b3 = d->b3;
    a.lambda_ce = lambda_ce;
    a.lambda_u = lambda_u;
    a.invP = 1.0f / (float)P;
    a.argmax = argmax;
    a.prob = prob;
    const int ntiles = (P + 127) / 128;
    if (target) {
        a.loss = loss; a.d_feat = d_feat; a.d_unc = d_unc;
        a.dW1 = dg->W1; a.db1 = dg->b1; a.dW2 = dg->W2; a.db2 = dg->b2; a.dW3 = dg->W3; a.db3 = dg->b3;
        // the loss and the weight gradients the kernel adds into, zeroed by one launch
        const ZeroList zl{{loss, dg->W1, dg->b1, dg->W2, dg->b2, dg->W3, dg->b3, loss_l1},
                          {2, kH1 * kD, kH1, kH2 * kH1, kH2, a.ncb * kH2, a.ncb, 1}};
        zero_list_kernel<<<img ? 8 : 7, 256, 0, s>>>(zl);
        LE_LAUNCHED();
        const size_t smem = train_smem(a.ncb);
        le_status st = set_smem(dec_train_kernel, smem);
        if (st != LE_OK) return st;
        const int grid = ntiles < sm_count() ? ntiles : sm_count();
        dec_train_kernel<<<grid, kTrainThreads, smem, s>>>(a);
        LE_LAUNCHED();
        return LE_OK;
    }
    const size_t smem = fwd_smem(a.ncb, 2);
    le_status st = set_smem(dec_fwd_kernel<2>, smem);
    if (st != LE_OK) return st;
    const int want = (ntiles + 1) / 2;
    const int grid = want < sm_count() ? want : sm_count();
    dec_fwd_kernel<2><<<grid, 256, smem, s>>>(a);
    LE_LAUNCHED();
    return LE_OK;
}

// W3's BF16 shared-memory image [n_cb x 128], Aq [16 x n_cb] FP32, G's BF16 image [n_cb x n_cb].
size_t query_fused_workspace(int32_t, int32_t n_cb, int32_t)
{
    return align_up(256ull * n_cb, 256) + align_up(sizeof(float) * 16 * n_cb, 256) + align_up(2ull * n_cb * n_cb, 256);
}

le_status query_fused(int32_t P, const float* feat, const le_decoder* d, const float* codebook, int32_t dd,
                      int32_t d_clip, const float* text, int32_t Q, const float* negs, int32_t n_neg, float* rel,
                      void* ws, size_t, cudaStream_t s)
{
    le_status st = check_fused_decoder(d, false);
    if (st != LE_OK) return st;
    const int ncb = d->n_cb;
    if (ncb % 64 != 0) {
        set_error("fused query needs n_cb to be a multiple of 64 (got %d)", ncb);
        return LE_ERR_UNSUPPORTED;
    }
    char* w = static_cast<char*>(ws);
    unsigned char* w3img = reinterpret_cast<unsigned char*>(w);
    float* Aq = reinterpret_cast<float*>(w + align_up(256ull * ncb, 256));
    unsigned char* img = reinterpret_cast<unsigned char*>(w + align_up(256ull * ncb, 256) +
                                                          align_up(sizeof(float) * 16 * ncb, 256));
    // G = S_c S_c^T (as the BF16 image) and Aq = [text; negs] S_c^T, FP32 on CUDA cores, one launch
    query_prep_kernel<<<dim3(ncb / 16, ncb / 16 + 1), 256, 0, s>>>(codebook, ncb, dd, d_clip, text, Q, negs, n_neg,
                                                                   img, Aq);
    LE_LAUNCHED();
    // W3's shared-memory image, reloaded after each tile when G's chunks 2-3 borrow its place (n_cb > 128)
    if (ncb > 128) {
        w3_image_kernel<<<16, 256, 0, s>>>(d->W3, ncb, w3img);
        LE_LAUNCHED();
    }
    DecArgs a{};
    a.P = P;
    a.ncb = ncb;
    a.feat = feat;
    a.W1 = d->W1; a.b1 = d->b1; a.W2 = d->W2; a.b2 = d->b2; a.W3 = d->W3; a.b3 = d->b3;
    a.G_img = img;
    a.W3_img = w3img;
    a.Aq = Aq;
    a.Q = Q;
    a.n_neg = n_neg;
    a.rel = rel;
    const size_t smem = query_smem(ncb);
    if ((st = set_smem(query_fused_kernel, smem)) != LE_OK) return st;
    const int ntiles = (P + 127) / 128;
    const int grid = ntiles < sm_count() ? ntiles : sm_count();
    query_fused_kernel<<<grid, 128 * kQueryParts, smem, s>>>(a);
    LE_LAUNCHED();
    return LE_OK;
}

le_status export_fused(int32_t P, const float* feat, const le_decoder* d, const float* codebook, int32_t dd,
                       __nv_bfloat16* out, void* ws, cudaStream_t s)
{
    le_status st = check_fused_decoder(d, false);
    if (st != LE_OK) return st;
    const int ncb = d->n_cb;
    unsigned char* img = static_cast<unsigned char*>(ws);
    unsigned char* w3img = img + (size_t)ncb * dd * 2;
    // output tensor map: [P rows, dd columns] BF16, boxes of 128 rows x 64 columns, 128-byte swizzle
    EncodeTiled enc;
    if ((st = tensor_map_encoder(&enc)) != LE_OK) return st;
    CUtensorMap tmap;
    const cuuint64_t dims[2] = {(cuuint64_t)dd, (cuuint64_t)P};
    const cuuint64_t strides[1] = {(cuuint64_t)dd * 2};
    const cuuint32_t box[2] = {64, 128};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, out, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed for the feature map");
        return LE_ERR_CUDA;
    }
    codebook_chunks_kernel<<<64, 256, 0, s>>>(codebook, ncb, dd, img);
    LE_LAUNCHED();
    DecArgs a{};
    a.P = P;
    a.ncb = ncb;
    a.feat = feat;
    a.W1 = d->W1; a.b1 = d->b1; a.W2 = d->W2; a.b2 = d->b2; a.W3 = d->W3; a.b3 = d->b3;
    a.G_img = img;
    a.dd = dd;
    a.fmap = out;
    a.w3_reload = export_stage_in_w3(ncb) ? 1 : 0;
    if (a.w3_reload && sbuf_bytes(ncb, 128) < 2 * kExportBox) {
        set_error("feature map export: no shared memory for the output staging with n_cb = %d", ncb);
        return LE_ERR_UNSUPPORTED;
    }
    if (a.w3_reload) {
        w3_image_kernel<<<16, 256, 0, s>>>(d->W3, ncb, w3img);
        LE_LAUNCHED();
        a.W3_img = w3img;
    }
    const size_t smem = export_smem(ncb);
    if ((st = set_smem(export_fused_kernel, smem)) != LE_OK) return st;
    const int ntiles = (P + 127) / 128;
    const int grid = ntiles < sm_count() ? ntiles : sm_count();
    export_fused_kernel<<<grid, 128 * kQueryParts, smem, s>>>(tmap, a);
    LE_LAUNCHED();
    return LE_OK;
}

}  // namespace leg

extern "C" le_status le_feature_map_workspace(int32_t n_cb, int32_t d, size_t* bytes)
{
    LE_TRACE("le_feature_map_workspace");
    LE_CHECK_ARG(bytes != nullptr, "bytes is null");
    LE_CHECK_ARG(n_cb > 0 && d > 0, "bad sizes");
    *bytes = (size_t)n_cb * d * 2 + (size_t)n_cb * 128 * 2;   // codebook image + W3 image
    return LE_OK;
}

extern "C" le_status le_feature_map(int32_t P, const float* feat, const le_decoder* dec, const float* codebook,
                                    int32_t d, uint16_t* out, void* workspace, size_t workspace_bytes, void* stream)
{
    LE_TRACE("le_feature_map");
    LE_CHECK_ARG(P >= 0, "P = %d < 0", P);
    LE_CHECK_ARG(dec != nullptr && codebook && workspace && (P == 0 || out), "null pointer");
    LE_CHECK_ARG(P == 0 || feat != nullptr, "null feat");
    LE_CHECK_ARG(leg::aligned16(out) && leg::aligned16(workspace), "out and workspace must be 16-byte aligned");
    if (d <= 0 || d % 64 != 0) {
        leg::set_error("feature map export needs d to be a positive multiple of 64 (got %d)", d);
        return LE_ERR_UNSUPPORTED;
    }
    LE_CHECK_ARG(workspace_bytes >= (size_t)dec->n_cb * d * 2 + (size_t)dec->n_cb * 128 * 2, "workspace too small");
    if (P == 0) return LE_OK;
    return leg::export_fused(P, feat, dec, codebook, d, reinterpret_cast<__nv_bfloat16*>(out), workspace,
                             leg::as_stream(stream));
}

extern "C" le_status le_selftest_bounded_wait(void* stream)
{
    LE_TRACE("le_selftest_bounded_wait");
    leg::selftest_wait_kernel<<<1, 32, 0, leg::as_stream(stream)>>>();
    LE_LAUNCHED();
    return LE_OK;
}

namespace leg {
le_status quant_take_timeout(bool* timed_out);
le_status smooth_take_timeout(bool* timed_out);
le_status wide_take_timeout(bool* timed_out);
}

extern "C" le_status le_device_status(void* stream)
{
    LE_TRACE("le_device_status");
    LE_CUDA(cudaStreamSynchronize(leg::as_stream(stream)));
    int flag = 0;
    LE_CUDA(cudaMemcpyFromSymbol(&flag, leg::g_tc_error, sizeof(int)));
    bool quant_flag = false;
    const le_status qs = leg::quant_take_timeout(&quant_flag);
    if (qs != LE_OK) return qs;
    bool smooth_flag = false;
    const le_status ss = leg::smooth_take_timeout(&smooth_flag);
    if (ss != LE_OK) return ss;
    bool wide_flag = false;
    const le_status ws = leg::wide_take_timeout(&wide_flag);
    if (ws != LE_OK) return ws;
    if ((quant_flag || smooth_flag || wide_flag) && !flag) {
        leg::set_error(quant_flag    ? "the quantisation kernel gave up on a bounded wait"
                       : smooth_flag ? "the smoothing kernel gave up on a bounded wait"
                                     : "a decoder kernel at the widths 8-128-256-N gave up on a bounded wait");
        return LE_ERR_TIMEOUT;
    }
    if (flag) {
        const int zero = 0;
        LE_CUDA(cudaMemcpyToSymbol(leg::g_tc_error, &zero, sizeof(int)));
        leg::set_error("a tensor-core kernel gave up on a bounded wait");
        return LE_ERR_TIMEOUT;
    }
    return LE_OK;
}
