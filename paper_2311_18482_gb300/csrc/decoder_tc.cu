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
//                     dL/dR_u, and the whole backward on the tensor cores.
//                     dL/dz, dL/dh2 and dL/dh1 are written once, pixel-major;
//                     the input-gradient MMAs read them K-major and the
//                     weight-gradient MMAs read the same buffers MN-major
//                     (contracting over the tile's pixels), with a ones column
//                     appended to each activation so the bias gradients come
//                     out of the same MMAs.  Weight gradients accumulate in
//                     TMEM over all tiles of a CTA and are flushed once.
//   query_fused_kernel relevancy (supp. Sec. "Inference", LERF): with
//                     p = softmax(z), |F_clip|^2 = p^T (S_c S_c^T) p and
//                     phi.q_j = p.(S_c q_j)/|F_clip|, so the 896-dim feature
//                     map F is never formed; S_c S_c^T (N x N) is streamed
//                     through shared memory in 64-column chunks with 1-D bulk
//                     async copies, S_c [q; n] sits in shared memory.
//
// Every mbarrier wait is bounded (about a second); on timeout the kernel
// records it in g_tc_error, stops issuing work, frees its TMEM and returns.
#include "tc_common.cuh"
#include "gemm_fp32.cuh"

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
    // query
    const unsigned char* G_img;     // ncb/64 chunks of [ncb x 64] canonical bf16
    const float* Aq;                // [16, ncb] fp32 = [text; negs] S_c^T
    int Q, n_neg;
    float* rel;
};

// Per-warpgroup state of the shared MLP front end.  With nhalf = 2 two
// warpgroups serve the same 128 TMEM lanes (rows) and split every epilogue
// by columns; `xch` is their shared-memory exchange for row-wide statistics.
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
    float4* xch;       // [2][128] (nhalf = 2 only)
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
__device__ bool mlp_forward(Front& f, const DecArgs& a, int p, bool valid)
{
    float v[16];
    if (f.half == 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = valid ? a.feat[(size_t)c * a.P + p] : 0.f;
        sbuf_store8(f.X1, f.tid, 0, v);
    }
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
#pragma unroll
        for (int s = 0; s < kH2 / 16; ++s)
            mma(f.tw, kdesc(f.H2, 0, 16 * s), kdesc(f.W3s, 0, 16 * s), idesc_bf16(a.ncb, false, false), s > 0);
        commit(f.mbar);
    }
    return wg_wait(f);
}

// Online max / argmax / log-sum-exp over the ncb logits in TMEM (+ b3); with
// two halves, each covers its columns and the pair combine through f.xch.
// Ties go to the lowest index.  zt = logit of class t (if t >= 0).
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
    if (f.nhalf == 2) {
        f.xch[f.half * 128 + f.tid] = make_float4(m, s, __int_as_float(am), zt);
        wg_sync(f);
        const float4 o = f.xch[(1 - f.half) * 128 + f.tid];
        wg_sync(f);
        const float m0 = f.half == 0 ? m : o.x, s0 = f.half == 0 ? s : o.y;
        const float m1 = f.half == 0 ? o.x : m, s1 = f.half == 0 ? o.y : s;
        const int a0 = f.half == 0 ? am : __float_as_int(o.z), a1 = f.half == 0 ? __float_as_int(o.z) : am;
        const bool t_mine = t >= c0 && t < c1;
        zt = t_mine ? zt : o.w;
        m = fmaxf(m0, m1);
        s = (m0 == -INFINITY ? 0.f : s0 * __expf(m0 - m)) + (m1 == -INFINITY ? 0.f : s1 * __expf(m1 - m));
        am = m1 > m0 ? a1 : a0;
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
// Training.  One CTA per SM, persistent over tiles; 256 threads: the two
// warpgroups serve the same 128 rows (TMEM lanes) and split each epilogue by
// columns.  TMEM: working 128 columns + the three weight-gradient accumulators.
constexpr uint32_t kAcc3 = 128, kAcc2 = 288, kAcc1 = 384;   // TMEM columns (32-aligned)
constexpr int kC1 = 16, kCH1 = 80, kCH2 = 144, kCD = 128;   // buffer widths (with ones columns)

__host__ constexpr size_t train_smem(int ncb)
{
    return weights_bytes(ncb) + sbuf_bytes(128, kC1) + sbuf_bytes(128, kCH1) + sbuf_bytes(128, kCH2) +
           3 * sbuf_bytes(128, kCD) + 2 * 128 * 16 + 128;
}

__global__ void __launch_bounds__(256, 1) dec_train_kernel(DecArgs a)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    Front f;
    unsigned char* p = load_weights(sm, a, f);
    f.X1 = SBuf{p, kC1};
    p += sbuf_bytes(128, kC1);
    f.H1 = SBuf{p, kCH1};
    p += sbuf_bytes(128, kCH1);
    f.H2 = SBuf{p, kCH2};
    p += sbuf_bytes(128, kCH2);
    const SBuf DZ{p, kCD}, DH2{p + sbuf_bytes(128, kCD), kCD}, DH1{p + 2 * sbuf_bytes(128, kCD), kCD};
    p += 3 * sbuf_bytes(128, kCD);
    f.xch = reinterpret_cast<float4*>(p);
    p += 2 * 128 * 16;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(p);
    uint32_t* slot = reinterpret_cast<uint32_t*>(p + 8);
    f.mbar = mbar;
    f.phase = 0;
    f.tid = threadIdx.x & 127;
    f.half = threadIdx.x >> 7;
    f.nhalf = 2;
    f.bar_id = 0;
    f.nthreads = blockDim.x;
    const int row = f.tid;
    const bool leader = threadIdx.x == 0;
    // constant columns of this row: ones for the bias gradients, zero padding
    {
        const float one[8] = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, zero[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (f.half == 0) {
            sbuf_store8(f.H1, row, 64, one);
            sbuf_store8(f.H1, row, 72, zero);
            sbuf_store8(f.H2, row, 128, one);
            sbuf_store8(f.H2, row, 136, zero);
        } else {
            for (int c = a.ncb; c < kCD; c += 8) sbuf_store8(DZ, row, c, zero);
            for (int c = 64; c < kCD; c += 8) sbuf_store8(DH1, row, c, zero);
        }
    }
    if (leader) mbar_init(mbar, 1);
    if (threadIdx.x < 32) tmem_alloc(slot, 512);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(slot);
    f.tw = tbase;
    f.lane = (uint32_t)(32 * (row >> 5)) << 16;

    const int ntiles = (a.P + 127) / 128;
    float acc_ce = 0.f, acc_u = 0.f;
    bool any = false;
    int c0, c1;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int px = tile * 128 + row;
        const bool valid = px < a.P;
        if (!mlp_forward(f, a, px, valid)) { any = false; break; }
        // softmax cross-entropy with uncertainty weighting (Eqs. 9-12)
        const float u = valid ? a.unc[px] : 0.f;
        const int t = valid ? a.target[px] : -1;
        float lse, zt;
        int am;
        logits_lse(f, a.ncb, lse, am, t, zt);
        const float ce = lse - zt;
        // dL/dz * P (1/P applied when the gradients are written)
        const float w = valid ? a.lambda_ce * (1.f - u) : 0.f;
        if (valid && f.half == 0) {
            a.d_unc[px] = (a.lambda_u - a.lambda_ce * ce) * a.invP;
            acc_ce += ce * (1.f - u);
            acc_u += u;
        }
        float v[16], h[16];
        my_cols(f, a.ncb, c0, c1);
        for (int c = c0; c < c1; c += 16) {
            tmem_ld16(f.tw + f.lane + c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = w * (__expf(v[j] + f.b3s[c + j] - lse) - (c + j == t ? 1.f : 0.f));
            sbuf_store8(DZ, row, c, v);
            sbuf_store8(DZ, row, c + 8, v + 8);
        }
        wg_publish(f);
        const uint32_t acc = any ? 1u : 0u;
        if (leader) {
            // dh2 = dz W3   (A = DZ K-major, B = W3 read MN-major)
            for (int s = 0; s < a.ncb / 16; ++s)
                mma(f.tw, kdesc(DZ, 0, 16 * s), mndesc(f.W3s, 16 * s, 0), idesc_bf16(kH2, false, true), s > 0);
            // dW3 | db3 += dz^T [h2 | 1]   (both read MN-major, contraction over pixels)
#pragma unroll
            for (int s = 0; s < 8; ++s)
                mma(tbase + kAcc3, mndesc(DZ, 16 * s, 0), mndesc(f.H2, 16 * s, 0), idesc_bf16(kCH2, true, true),
                    s > 0 ? 1u : acc);
            commit(f.mbar);
        }
        if (!wg_wait(f)) { any = false; break; }
        // dh2 * [h2 > 0]
        my_cols(f, kH2, c0, c1);
        for (int c = c0; c < c1; c += 16) {
            tmem_ld16(f.tw + f.lane + c, v);
            sbuf_load8(f.H2, row, c, h);
            sbuf_load8(f.H2, row, c + 8, h + 8);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = h[j] > 0.f ? v[j] : 0.f;
            sbuf_store8(DH2, row, c, v);
            sbuf_store8(DH2, row, c + 8, v + 8);
        }
        wg_publish(f);
        if (leader) {
#pragma unroll
            for (int s = 0; s < kH2 / 16; ++s)
                mma(f.tw, kdesc(DH2, 0, 16 * s), mndesc(f.W2s, 16 * s, 0), idesc_bf16(kH1, false, true), s > 0);
#pragma unroll
            for (int s = 0; s < 8; ++s)
                mma(tbase + kAcc2, mndesc(DH2, 16 * s, 0), mndesc(f.H1, 16 * s, 0), idesc_bf16(kCH1, true, true),
                    s > 0 ? 1u : acc);
            commit(f.mbar);
        }
        if (!wg_wait(f)) { any = false; break; }
        // dh1 * [h1 > 0]
        my_cols(f, kH1, c0, c1);
        for (int c = c0; c < c1; c += 16) {
            tmem_ld16(f.tw + f.lane + c, v);
            sbuf_load8(f.H1, row, c, h);
            sbuf_load8(f.H1, row, c + 8, h + 8);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = h[j] > 0.f ? v[j] : 0.f;
            sbuf_store8(DH1, row, c, v);
            sbuf_store8(DH1, row, c + 8, v + 8);
        }
        wg_publish(f);
        if (leader) {
#pragma unroll
            for (int s = 0; s < kH1 / 16; ++s)
                mma(f.tw, kdesc(DH1, 0, 16 * s), mndesc(f.W1s, 16 * s, 0), idesc_bf16(16, false, true), s > 0);
#pragma unroll
            for (int s = 0; s < 8; ++s)
                mma(tbase + kAcc1, mndesc(DH1, 16 * s, 0), mndesc(f.X1, 16 * s, 0), idesc_bf16(16, true, true),
                    s > 0 ? 1u : acc);
            commit(f.mbar);
        }
        if (!wg_wait(f)) { any = false; break; }
        any = true;
        if (f.half == 0) {
            tmem_ld16(f.tw + f.lane, v);
            if (valid)
#pragma unroll
                for (int c = 0; c < kD; ++c) a.d_feat[(size_t)c * a.P + px] = v[c] * a.invP;
        }
        fence_before();
        __syncthreads();
    }
    // flush the weight-gradient accumulators (row = this thread's TMEM lane, columns split by half)
    if (any) {
        float v[16];
        my_cols(f, kCH2, c0, c1);
        for (int c = c0; c < c1; c += 16) {
            tmem_ld16(tbase + kAcc3 + f.lane + c, v);
            if (row < a.ncb)
                for (int j = 0; j < 16; ++j) {
                    const int col = c + j;
                    if (col < kH2) atomicAdd(a.dW3 + (size_t)row * kH2 + col, v[j] * a.invP);
                    else if (col == kH2) atomicAdd(a.db3 + row, v[j] * a.invP);
                }
        }
        my_cols(f, kCH1, c0, c1);
        for (int c = c0; c < c1; c += 16) {
            tmem_ld16(tbase + kAcc2 + f.lane + c, v);
            for (int j = 0; j < 16; ++j) {
                const int col = c + j;
                if (col < kH1) atomicAdd(a.dW2 + (size_t)row * kH1 + col, v[j] * a.invP);
                else if (col == kH1) atomicAdd(a.db2 + row, v[j] * a.invP);
            }
        }
        if (f.half == 0) {
            tmem_ld16(tbase + kAcc1 + f.lane, v);
            if (row < kH1) {
                for (int j = 0; j < kD; ++j) atomicAdd(a.dW1 + (size_t)row * kD + j, v[j] * a.invP);
                atomicAdd(a.db1 + row, v[kD] * a.invP);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_ce += __shfl_xor_sync(0xffffffffu, acc_ce, o);
        acc_u += __shfl_xor_sync(0xffffffffu, acc_u, o);
    }
    if ((threadIdx.x & 31) == 0 && f.half == 0) {
        atomicAdd(a.loss, acc_ce * a.invP);
        atomicAdd(a.loss + 1, acc_u * a.invP);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (threadIdx.x < 32) tmem_dealloc(tbase, 512);
}

// ---------------------------------------------------------------------------
// Query: decode, softmax, relevancy.  One warpgroup per CTA; TMEM: logits in
// [0, ncb) (later the 16 text/negative projections in [0, 16)), p^T G in
// [256, 256 + ncb).  The activations X1/H1/H2 and the BF16 softmax P share one
// region (P is written after the last MMA that reads H2 has completed).
constexpr uint32_t kTG = 256;

__host__ constexpr size_t query_smem(int ncb)
{
    return weights_bytes(ncb) + sbuf_bytes(16, ncb) +
           (sbuf_bytes(128, ncb) > kFwdWgBytes ? sbuf_bytes(128, ncb) : kFwdWgBytes) + 2 * sbuf_bytes(ncb, 64) + 128;
}

__global__ void __launch_bounds__(128, 1) query_fused_kernel(DecArgs a)
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
    p += sbuf_bytes(128, a.ncb) > kFwdWgBytes ? sbuf_bytes(128, a.ncb) : kFwdWgBytes;
    const uint32_t chunk_bytes = sbuf_bytes(a.ncb, 64);
    const SBuf Gs[2] = {SBuf{p, 64}, SBuf{p + chunk_bytes, 64}};
    p += 2 * chunk_bytes;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(p);     // [0] MMA, [1], [2] G slots
    uint32_t* slot = reinterpret_cast<uint32_t*>(p + 24);
    const int tid = threadIdx.x;
    sbuf_fill(Aqs, 16, a.Aq, a.ncb, 16, a.ncb);
    f.mbar = mbar;
    f.phase = 0;
    f.tid = tid;
    f.bar_id = 0;
    f.nthreads = blockDim.x;
    f.half = 0;
    f.nhalf = 1;
    f.xch = nullptr;
    if (tid == 0)
        for (int i = 0; i < 3; ++i) mbar_init(mbar + i, 1);
    if (tid < 32) tmem_alloc(slot, 512);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tbase = *reinterpret_cast<volatile uint32_t*>(slot);
    f.tw = tbase;
    f.lane = (uint32_t)(32 * (tid >> 5)) << 16;
    const int nch = a.ncb / 64;                 // G chunks (64 K-columns each)
    uint32_t gphase[2] = {0u, 0u};
    bool pending[2] = {false, false};          // a load into the slot is in flight (thread 0 only)
    auto load_chunk = [&](int kc, int s) {
        mbar_expect_tx(mbar + 1 + s, chunk_bytes);
        bulk_g2s(Gs[s].p, a.G_img + (size_t)kc * chunk_bytes, chunk_bytes, mbar + 1 + s);
        pending[s] = true;
    };
    const int ntiles = (a.P + 127) / 128;
    bool ok = true;
    if (tid == 0 && blockIdx.x < ntiles)
        for (int s = 0; s < 2 && s < nch; ++s) load_chunk(s, s);
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int px = tile * 128 + tid;
        const bool valid = px < a.P;
        if (!mlp_forward(f, a, px, valid)) break;
        float lse, zt, v[16];
        int am;
        logits_lse(f, a.ncb, lse, am, -1, zt);
        for (int c = 0; c < a.ncb; c += 16) {
            tmem_ld16(f.tw + f.lane + c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __expf(v[j] + f.b3s[c + j] - lse);
            sbuf_store8(Ps, tid, c, v);
            sbuf_store8(Ps, tid, c + 8, v + 8);
        }
        wg_publish(f);
        // p . (S_c [q; n]) into [0, 16), p^T G into [256, 256 + ncb), G chunk by chunk
        bool tmo = false;
        for (int kc0 = 0; kc0 < nch; kc0 += 2) {
            if (tid == 0) {
                if (kc0 == 0)
                    for (int s = 0; s < a.ncb / 16; ++s)
                        mma(tbase, kdesc(Ps, 0, 16 * s), kdesc(Aqs, 0, 16 * s), idesc_bf16(16, false, false), s > 0);
                for (int s = 0; s < 2 && kc0 + s < nch; ++s) {
                    if (!mbar_wait(mbar + 1 + s, gphase[s])) tmo = true;
                    gphase[s] ^= 1u;
                    pending[s] = false;
                    for (int k = 0; k < 4; ++k)
                        mma(tbase + kTG, kdesc(Ps, 0, 64 * (kc0 + s) + 16 * k), kdesc(Gs[s], 0, 16 * k),
                            idesc_bf16(a.ncb, false, false), (kc0 + s) > 0 || k > 0);
                }
                commit(f.mbar);
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
        }
        if (!ok) break;
        // relevancy
        float ptgp = 0.f, pp[16];
        for (int c = 0; c < a.ncb; c += 16) {
            tmem_ld16(tbase + kTG + f.lane + c, v);
            sbuf_load8(Ps, tid, c, pp);
            sbuf_load8(Ps, tid, c + 8, pp + 8);
#pragma unroll
            for (int j = 0; j < 16; ++j) ptgp = fmaf(pp[j], v[j], ptgp);
        }
        tmem_ld16(tbase + f.lane, v);
        const float inv = rsqrtf(fmaxf(ptgp, 1e-30f));
        float smax = -INFINITY;
        for (int j = a.Q; j < a.Q + a.n_neg; ++j) smax = fmaxf(smax, v[j] * inv);
        if (valid)
            for (int j = 0; j < a.Q; ++j) a.rel[(size_t)j * a.P + px] = 1.f / (1.f + __expf(smax - v[j] * inv));
        fence_before();
        __syncthreads();
    }
    // drain copies still in flight (only after an early exit) before the shared memory goes away
    if (tid == 0)
        for (int s = 0; s < 2; ++s)
            if (pending[s]) mbar_wait(mbar + 1 + s, gphase[s]);
    fence_before();
    __syncthreads();
    fence_after();
    if (tid < 32) tmem_dealloc(tbase, 512);
}

// G = S_c S_c^T (fp32) -> chunked canonical bf16 image: chunk kc holds columns
// [64 kc, 64 kc + 64) of every row, as an [ncb x 64] canonical buffer.
__global__ void gram_layout_kernel(const float* __restrict__ G, int ncb, unsigned char* __restrict__ img)
{
    const int n8 = ncb * (ncb / 8);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n8; i += gridDim.x * blockDim.x) {
        const int r = i / (ncb / 8), c0 = (i % (ncb / 8)) * 8;
        const int kc = c0 / 64, cc = c0 % 64;
        __nv_bfloat162 h[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(G[(size_t)r * ncb + c0 + 2 * j], G[(size_t)r * ncb + c0 + 2 * j + 1]);
        unsigned char* dst = img + (size_t)kc * ncb * 64 * 2 + ((r >> 3) * 8 * 128 + (cc >> 3) * 128 + (r & 7) * 16);
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<uint4*>(h);
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

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
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
                       const le_decoder_grads* dg, int32_t* argmax, float* prob, void*, size_t, cudaStream_t s)
{
    DecArgs a{};
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
        LE_CUDA(cudaMemsetAsync(loss, 0, 2 * sizeof(float), s));
        LE_CUDA(cudaMemsetAsync(dg->W1, 0, sizeof(float) * kH1 * kD, s));
        LE_CUDA(cudaMemsetAsync(dg->b1, 0, sizeof(float) * kH1, s));
        LE_CUDA(cudaMemsetAsync(dg->W2, 0, sizeof(float) * kH2 * kH1, s));
        LE_CUDA(cudaMemsetAsync(dg->b2, 0, sizeof(float) * kH2, s));
        LE_CUDA(cudaMemsetAsync(dg->W3, 0, sizeof(float) * a.ncb * kH2, s));
        LE_CUDA(cudaMemsetAsync(dg->b3, 0, sizeof(float) * a.ncb, s));
        const size_t smem = train_smem(a.ncb);
        le_status st = set_smem(dec_train_kernel, smem);
        if (st != LE_OK) return st;
        const int grid = ntiles < sm_count() ? ntiles : sm_count();
        dec_train_kernel<<<grid, 256, smem, s>>>(a);
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

size_t query_fused_workspace(int32_t, int32_t n_cb, int32_t)
{
    return align_up(sizeof(float) * n_cb * n_cb, 256) + align_up(sizeof(float) * 16 * n_cb, 256) +
           align_up(2ull * n_cb * n_cb, 256);
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
    float* G = reinterpret_cast<float*>(w);
    float* Aq = reinterpret_cast<float*>(w + align_up(sizeof(float) * ncb * ncb, 256));
    unsigned char* img = reinterpret_cast<unsigned char*>(w + align_up(sizeof(float) * ncb * ncb, 256) +
                                                          align_up(sizeof(float) * 16 * ncb, 256));
    // G = S_c S_c^T and Aq = [text; negs] S_c^T, FP32 on CUDA cores (small, once per call)
    GemmArgs g{};
    g.M = ncb; g.N = ncb; g.K = d_clip;
    g.A = codebook; g.lda = dd; g.B = codebook; g.ldb = dd; g.C = G; g.ldc = ncb;
    if ((st = sgemm(false, true, g, 1, s)) != LE_OK) return st;
    LE_CUDA(cudaMemsetAsync(Aq, 0, sizeof(float) * 16 * ncb, s));
    g = GemmArgs{};
    g.M = Q; g.N = ncb; g.K = d_clip;
    g.A = text; g.lda = d_clip; g.B = codebook; g.ldb = dd; g.C = Aq; g.ldc = ncb;
    if ((st = sgemm(false, true, g, 1, s)) != LE_OK) return st;
    g.M = n_neg; g.A = negs; g.C = Aq + (size_t)Q * ncb;
    if ((st = sgemm(false, true, g, 1, s)) != LE_OK) return st;
    gram_layout_kernel<<<64, 256, 0, s>>>(G, ncb, img);
    LE_LAUNCHED();
    DecArgs a{};
    a.P = P;
    a.ncb = ncb;
    a.feat = feat;
    a.W1 = d->W1; a.b1 = d->b1; a.W2 = d->W2; a.b2 = d->b2; a.W3 = d->W3; a.b3 = d->b3;
    a.G_img = img;
    a.Aq = Aq;
    a.Q = Q;
    a.n_neg = n_neg;
    a.rel = rel;
    const size_t smem = query_smem(ncb);
    if ((st = set_smem(query_fused_kernel, smem)) != LE_OK) return st;
    const int ntiles = (P + 127) / 128;
    const int grid = ntiles < sm_count() ? ntiles : sm_count();
    query_fused_kernel<<<grid, 128, smem, s>>>(a);
    LE_LAUNCHED();
    return LE_OK;
}

}  // namespace leg

extern "C" le_status le_selftest_bounded_wait(void* stream)
{
    leg::selftest_wait_kernel<<<1, 32, 0, leg::as_stream(stream)>>>();
    LE_LAUNCHED();
    return LE_OK;
}

extern "C" le_status le_device_status(void* stream)
{
    LE_CUDA(cudaStreamSynchronize(leg::as_stream(stream)));
    int flag = 0;
    LE_CUDA(cudaMemcpyFromSymbol(&flag, leg::g_tc_error, sizeof(int)));
    if (flag) {
        const int zero = 0;
        LE_CUDA(cudaMemcpyToSymbol(leg::g_tc_error, &zero, sizeof(int)));
        leg::set_error("a tensor-core kernel gave up on a bounded wait");
        return LE_ERR_TIMEOUT;
    }
    return LE_OK;
}
