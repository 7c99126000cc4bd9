// Adaptive spatial smoothing (Sec. 3.4, Eqs. eq:lem_fmlp and eq:lem_loss_mlp;
// supplementary Tab. pemlp): per Gaussian s_MLP = MLP(p) (positional encoding
// of frequency 0 = the position), MLP 3 -> 128 -> 128 -> 128 -> 8 (ReLU x 3),
//   L_smo = |s_MLP - s_G*| + max(u*, w_s) |s_MLP* - s_G|   (* = stop gradient),
// its mean over the Gaussians times lambda_smo, the gradient of every MLP
// parameter (through the first term) and of s_G (through the second).
//
// smooth_kernel: persistent, one CTA per SM, tiles of 128 Gaussians one after
// another.  Four warpgroups serve the tile's 128 rows (TMEM lanes), each
// taking 32 of every 128-column epilogue's columns; the loss epilogue is
// warpgroup 0's.  Thread 0 issues each tcgen05.mma round; after it completes,
// all threads run its epilogue (bias, ReLU and its mask, BF16 into shared
// memory):
//   forward  H1 = relu(X W1^T + b1), H2, H3, Z = H3 W4^T + b4 (FP32 accumulation)
//   loss     per row: diff = Z - s_G, n = |diff|; dZ = lambda/n_total diff/n;
//            d_feat -= lambda/n_total max(u, w_s) diff/n (added to the caller's array)
//   backward dH3 = (dZ W4) o [H3 > 0], dH2 = (dH3 W3) o [H2 > 0], dH1 = ...;
//            each dH overwrites its H in shared memory once the MMAs that read
//            H have completed.  Weight gradients dW = dH^T H_prev accumulate in
//            TMEM over all of a CTA's tiles (MMAs reading both operands
//            MN-major from the row-major activation buffers, no transposed
//            copies); the bias sums come from MMAs against a ones column (b2, b3),
//            the ones column of X (b1) and a warp transposition (b4).
// At the end each CTA adds its accumulators to the caller's gradients with
// atomics.  Every wait is bounded; on a timeout the kernel records it,
// stops issuing work, waits (bounded) for its MMAs and frees its TMEM.
#include "tc_common.cuh"

namespace leg {

__device__ int g_smooth_error;

namespace {
using namespace tc;

constexpr int kH = 128, kS = 8;
constexpr int kParts = 4;                    // warpgroups per CTA
constexpr int kThreadsS = 128 * kParts;
// TMEM columns
constexpr uint32_t kAcc = 0, kDW2 = 128, kDW3 = 256, kDW1 = 384, kDW4 = 400, kDB2 = 416, kDB3 = 432;

struct SmoothArgs {
    int n, ntiles;
    const float *means, *feat, *unc;
    const float *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;
    float w_s, scale;              // scale = lambda_smo / n
    float* loss;
    float* d_feat;
    int d_feat_stride;
    float* s_mlp;                  // nullable
    float *dW1, *db1, *dW2, *db2, *dW3, *db3, *dW4, *db4;
};

// Shared-memory plan (canonical no-swizzle BF16 buffers; byte offsets).
constexpr uint32_t kOW1 = 0;                                 // [128][16]
constexpr uint32_t kOW2 = kOW1 + sbuf_bytes(128, 16);        // [128][128]
constexpr uint32_t kOW3 = kOW2 + sbuf_bytes(128, 128);
constexpr uint32_t kOW4 = kOW3 + sbuf_bytes(128, 128);       // [16][128]
constexpr uint32_t kOX = kOW4 + sbuf_bytes(16, 128);         // [128][16], column 3 = 1
constexpr uint32_t kOH1 = kOX + sbuf_bytes(128, 16);         // [128][128] H1, later dH1
constexpr uint32_t kOH2 = kOH1 + sbuf_bytes(128, 128);
constexpr uint32_t kOH3 = kOH2 + sbuf_bytes(128, 128);
constexpr uint32_t kODZ = kOH3 + sbuf_bytes(128, 128);       // [128][16]
constexpr uint32_t kOE = kODZ + sbuf_bytes(128, 16);         // [128][16], column 0 = 1
constexpr uint32_t kOB = kOE + sbuf_bytes(128, 16);          // biases FP32: b1, b2, b3 (128 each), b4 (8)
constexpr uint32_t kOM = kOB + (3 * kH + 16) * 4;           // ReLU masks: [3 layers][4 words][128 rows] u32
constexpr uint32_t kOBar = kOM + 3 * 4 * 128 * 4;
constexpr uint32_t kSmoothSmem = kOBar + 32 + 1024;

struct Ctx {
    unsigned char* sm;
    uint32_t s0;                   // shared address of sm
    uint64_t* bar;
    uint32_t* tslot;
    uint32_t phase;
    uint32_t tmem, lanef;
    int row;
    int part;                      // warpgroup: columns [32 part, 32 part + 32) of each hidden epilogue
};

// Wait for the MMA round just committed; every thread agrees on the outcome.
__device__ __forceinline__ bool round_wait(Ctx& c)
{
    const bool ok = mbar_wait(c.bar, c.phase);
    c.phase ^= 1u;
    const bool bad = __syncthreads_or(!ok);
    fence_after();
    return !bad;
}

// Shared-memory writes visible to the tensor core, TMEM reads ordered before the next MMAs.
__device__ __forceinline__ void publish()
{
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
}

// This warpgroup's 32 columns of the epilogue of a 128-column hidden layer:
// v = acc + b; relu; BF16 into H; the ReLU mask bits into mask[part * 128 + row].
__device__ __forceinline__ void hidden_epilogue(const Ctx& c, const float* b, uint32_t hoff, uint32_t* mask)
{
    const SBuf Hs{c.sm + hoff, kH};
    {
        const int q = 2 * c.part;
        uint32_t mw = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[16];
            tmem_ld16(c.tmem + c.lanef + kAcc + 16 * (q + h), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float x = v[j] + b[16 * (q + h) + j];
                mw |= (x > 0.f ? 1u : 0u) << (16 * h + j);
                v[j] = fmaxf(x, 0.f);
            }
            sbuf_store8(Hs, c.row, 16 * (q + h), v);
            sbuf_store8(Hs, c.row, 16 * (q + h) + 8, v + 8);
        }
        mask[(q >> 1) * 128 + c.row] = mw;
    }
}

// This warpgroup's 32 columns of a backward epilogue: dH = acc o mask, BF16 into H's buffer.
__device__ __forceinline__ void grad_epilogue(const Ctx& c, uint32_t hoff, const uint32_t* mask)
{
    const SBuf Hs{c.sm + hoff, kH};
    {
        const int q = 2 * c.part;
        const uint32_t mw = mask[(q >> 1) * 128 + c.row];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v[16];
            tmem_ld16(c.tmem + c.lanef + kAcc + 16 * (q + h), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = ((mw >> (16 * h + j)) & 1u) ? v[j] : 0.f;
            sbuf_store8(Hs, c.row, 16 * (q + h), v);
            sbuf_store8(Hs, c.row, 16 * (q + h) + 8, v + 8);
        }
    }
}

// K-major descriptor of a C-column buffer at shared offset off (rows from 0).
__device__ __forceinline__ uint64_t kd(uint32_t s0, uint32_t off, int C) { return kdesc_at(s0 + off, C, 0, 0); }
// MN-major descriptor (rows = K) of a C-column buffer.
__device__ __forceinline__ uint64_t md(uint32_t s0, uint32_t off, int C) { return mndesc_at(s0 + off, C, 0, 0); }

// One MMA round, issued by thread 0.  K steps of 16 move the start address by
// 16 units (K-major) or 2C units (MN-major over a C-column buffer).  The
// arguments come by value, so the caller's context stays in registers.
__device__ __noinline__ void issue(uint32_t s0, uint32_t t, uint64_t* bar, int round, bool first_tile)
{
    const uint32_t keep = first_tile ? 0u : 1u;
    switch (round) {
        case 0:   // H1 pre-activation = X W1^T
            mma(t + kAcc, kd(s0, kOX, 16), kd(s0, kOW1, 16), idesc_bf16(kH, false, false), 0u);
            break;
        case 1:   // H2 = H1 W2^T
        case 2: { // H3 = H2 W3^T
            const uint64_t a = kd(s0, round == 1 ? kOH1 : kOH2, kH), b = kd(s0, round == 1 ? kOW2 : kOW3, kH);
#pragma unroll
            for (int k = 0; k < 8; ++k) mma(t + kAcc, a + 16 * k, b + 16 * k, idesc_bf16(kH, false, false), k > 0);
            break;
        }
        case 3: { // Z = H3 W4^T (N = 16, 8 used)
            const uint64_t a = kd(s0, kOH3, kH), b = kd(s0, kOW4, kH);
#pragma unroll
            for (int k = 0; k < 8; ++k) mma(t + kAcc, a + 16 * k, b + 16 * k, idesc_bf16(16, false, false), k > 0);
            break;
        }
        case 4: { // dH3 (pre-mask) = dZ W4; dW4^T += H3^T dZ
            mma(t + kAcc, kd(s0, kODZ, 16), md(s0, kOW4, kH), idesc_bf16(kH, false, true), 0u);
            const uint64_t a = md(s0, kOH3, kH), b = md(s0, kODZ, 16);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                mma(t + kDW4, a + 256 * k, b + 32 * k, idesc_bf16(16, true, true), k > 0 ? 1u : keep);
            break;
        }
        case 5:   // dH2 = dH3 W3; dW3 += dH3^T H2; db3 += dH3^T 1
        case 6: { // dH1 = dH2 W2; dW2 += dH2^T H1; db2 += dH2^T 1
            const uint32_t dh = round == 5 ? kOH3 : kOH2, w = round == 5 ? kOW3 : kOW2, hp = round == 5 ? kOH2 : kOH1;
            const uint32_t dw = round == 5 ? kDW3 : kDW2, db = round == 5 ? kDB3 : kDB2;
            const uint64_t ak = kd(s0, dh, kH), wm = md(s0, w, kH);
#pragma unroll
            for (int k = 0; k < 8; ++k) mma(t + kAcc, ak + 16 * k, wm + 256 * k, idesc_bf16(kH, false, true), k > 0);
            const uint64_t am = md(s0, dh, kH), hm = md(s0, hp, kH), em = md(s0, kOE, 16);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                mma(t + dw, am + 256 * k, hm + 256 * k, idesc_bf16(kH, true, true), k > 0 ? 1u : keep);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                mma(t + db, am + 256 * k, em + 32 * k, idesc_bf16(16, true, true), k > 0 ? 1u : keep);
            break;
        }
        default: { // dW1 (+ db1 in column 3) += dH1^T X
            const uint64_t am = md(s0, kOH1, kH), xm = md(s0, kOX, 16);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                mma(t + kDW1, am + 256 * k, xm + 32 * k, idesc_bf16(16, true, true), k > 0 ? 1u : keep);
            break;
        }
    }
    commit(bar);
}

// Sum over the warp's 32 rows of 16 values (recursive halving); lanes 2j, 2j+1 hold column j.
template <int N, int O>
__device__ __forceinline__ void halve16(float* v, bool upper)
{
    constexpr int Hh = N / 2;
#pragma unroll
    for (int i = 0; i < Hh; ++i) {
        const float lo = v[i], hi = v[i + Hh];
        const float recv = __shfl_xor_sync(0xffffffffu, upper ? lo : hi, O);
        v[i] = (upper ? hi : lo) + recv;
    }
}

__device__ __forceinline__ float colsum16(float* v, int lane)
{
    halve16<16, 16>(v, lane & 16);
    halve16<8, 8>(v, lane & 8);
    halve16<4, 4>(v, lane & 4);
    halve16<2, 2>(v, lane & 2);
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__global__ void __launch_bounds__(kThreadsS, 1) smooth_kernel(SmoothArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    Ctx c;
    c.sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    c.s0 = smem_u32(c.sm);
    c.bar = reinterpret_cast<uint64_t*>(c.sm + kOBar);
    c.tslot = reinterpret_cast<uint32_t*>(c.sm + kOBar + 16);
    c.phase = 0;
    c.row = threadIdx.x & 127;
    c.part = threadIdx.x >> 7;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    c.lanef = (uint32_t)(32 * (warp & 3)) << 16;
    // weights (BF16, [out][in]), biases (FP32), the ones operand
    sbuf_fill(SBuf{c.sm + kOW1, 16}, 128, a.W1, 3, kH, 3);
    sbuf_fill(SBuf{c.sm + kOW2, kH}, 128, a.W2, kH, kH, kH);
    sbuf_fill(SBuf{c.sm + kOW3, kH}, 128, a.W3, kH, kH, kH);
    sbuf_fill(SBuf{c.sm + kOW4, kH}, 16, a.W4, kH, kS, kH);
    float* bs = reinterpret_cast<float*>(c.sm + kOB);
    for (int i = threadIdx.x; i < 3 * kH + 16; i += blockDim.x)
        bs[i] = i < kH ? a.b1[i] : i < 2 * kH ? a.b2[i - kH] : i < 3 * kH ? a.b3[i - 2 * kH]
              : (i - 3 * kH < kS ? a.b4[i - 3 * kH] : 0.f);
    if (c.part == 0) {
        float v[8] = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        sbuf_store8(SBuf{c.sm + kOE, 16}, c.row, 0, v);
        sbuf_store8(SBuf{c.sm + kOE, 16}, c.row, 8, z);
    }
    if (threadIdx.x == 0) mbar_init(c.bar, 1);
    if (warp == 0) tmem_alloc(c.tslot, 512);
    fence_proxy_async();
    fence_before();
    __syncthreads();
    fence_after();
    c.tmem = *reinterpret_cast<volatile uint32_t*>(c.tslot);

    const float* b1 = bs;
    const float* b2 = bs + kH;
    const float* b3 = bs + 2 * kH;
    const float* b4 = bs + 3 * kH;
    float lsum = 0.f, db4acc = 0.f;
    bool ok = true, any = false;
    for (int t = blockIdx.x; t < a.ntiles && ok; t += gridDim.x) {
        const bool first = !any;
        any = true;
        const int g = t * 128 + c.row;
        const bool valid = g < a.n;
        const bool p0 = c.part == 0;             // warpgroup 0: the row's inputs, X and the loss
        // this row's s_G, u and current d_feat, loaded now so that the forward rounds hide their latency
        float fg[kS], df[kS], ug = 0.f;
        if (valid && p0) {
            const float4 f0 = reinterpret_cast<const float4*>(a.feat)[2 * (size_t)g];
            const float4 f1 = reinterpret_cast<const float4*>(a.feat)[2 * (size_t)g + 1];
            fg[0] = f0.x; fg[1] = f0.y; fg[2] = f0.z; fg[3] = f0.w;
            fg[4] = f1.x; fg[5] = f1.y; fg[6] = f1.z; fg[7] = f1.w;
            ug = a.unc[g];
#pragma unroll
            for (int k = 0; k < kS; ++k) df[k] = a.d_feat[(size_t)g * a.d_feat_stride + k];
        } else {
#pragma unroll
            for (int k = 0; k < kS; ++k) fg[k] = df[k] = 0.f;
        }
        if (p0) {   // X = [p, 1, 0...]
            float v[8] = {0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 0.f}, z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (valid) {
                v[0] = a.means[3 * (size_t)g];
                v[1] = a.means[3 * (size_t)g + 1];
                v[2] = a.means[3 * (size_t)g + 2];
            }
            sbuf_store8(SBuf{c.sm + kOX, 16}, c.row, 0, v);
            sbuf_store8(SBuf{c.sm + kOX, 16}, c.row, 8, z);
        }
        uint32_t* m1 = reinterpret_cast<uint32_t*>(c.sm + kOM);
        uint32_t* m2 = m1 + 4 * 128;
        uint32_t* m3 = m2 + 4 * 128;
        publish();
        if (threadIdx.x == 0) issue(c.s0, c.tmem, c.bar, 0, first);
        if (!(ok = round_wait(c))) break;
        hidden_epilogue(c, b1, kOH1, m1);
        publish();
        if (threadIdx.x == 0) issue(c.s0, c.tmem, c.bar, 1, first);
        if (!(ok = round_wait(c))) break;
        hidden_epilogue(c, b2, kOH2, m2);
        publish();
        if (threadIdx.x == 0) issue(c.s0, c.tmem, c.bar, 2, first);
        if (!(ok = round_wait(c))) break;
        hidden_epilogue(c, b3, kOH3, m3);
        publish();
        if (threadIdx.x == 0) issue(c.s0, c.tmem, c.bar, 3, first);
        if (!(ok = round_wait(c))) break;
        if (p0) {   // loss and the output gradient
            float z[16];
            tmem_ld16(c.tmem + c.lanef + kAcc, z);
            float diff[kS], nn = 0.f;
#pragma unroll
            for (int k = 0; k < kS; ++k) {
                const float s = z[k] + b4[k];
                if (valid && a.s_mlp) a.s_mlp[(size_t)g * kS + k] = s;
                diff[k] = valid ? s - fg[k] : 0.f;
                nn = fmaf(diff[k], diff[k], nn);
            }
            nn = sqrtf(nn);
            const float wgt = valid ? fmaxf(ug, a.w_s) : 0.f;
            lsum += (1.f + wgt) * nn;
            const float inv = nn > 0.f ? a.scale / nn : 0.f;
            float dz[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) dz[k] = k < kS ? diff[k] * inv : 0.f;
            if (valid)
#pragma unroll
                for (int k = 0; k < kS; ++k) a.d_feat[(size_t)g * a.d_feat_stride + k] = df[k] - wgt * dz[k];
            sbuf_store8(SBuf{c.sm + kODZ, 16}, c.row, 0, dz);
            sbuf_store8(SBuf{c.sm + kODZ, 16}, c.row, 8, dz + 8);
            db4acc += colsum16(dz, lane);       // lanes 2k, 2k+1: column k (k < 8)
        }
        publish();
        if (threadIdx.x == 0) issue(c.s0, c.tmem, c.bar, 4, first);
        if (!(ok = round_wait(c))) break;
        grad_epilogue(c, kOH3, m3);              // dH3 over H3 (read by dW4, complete)
        publish();
        if (threadIdx.x == 0) issue(c.s0, c.tmem, c.bar, 5, first);
        if (!(ok = round_wait(c))) break;
        grad_epilogue(c, kOH2, m2);              // dH2 over H2
        publish();
        if (threadIdx.x == 0) issue(c.s0, c.tmem, c.bar, 6, first);
        if (!(ok = round_wait(c))) break;
        grad_epilogue(c, kOH1, m1);              // dH1 over H1
        publish();
        if (threadIdx.x == 0) issue(c.s0, c.tmem, c.bar, 7, first);
        if (!(ok = round_wait(c))) break;
    }
    if (!ok) {
        if (threadIdx.x == 0) {
            atomicExch(&g_smooth_error, 1);
            // nothing of ours may still be running when TMEM is freed
            commit(c.bar);
            (void)mbar_wait(c.bar, c.phase);
        }
    } else if (any) {
        // flush: TMEM lane = this thread's row of each accumulator
        // flush: TMEM lane = this thread's row of each accumulator; warpgroup p takes
        // columns [32 p, 32 p + 32) of dW2 and dW3 and one of the small blocks
        float v[16];
        const int r = c.row;
#pragma unroll
        for (int q = 2 * c.part; q < 2 * c.part + 2; ++q) {
            tmem_ld16(c.tmem + c.lanef + kDW2 + 16 * q, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) atomicAdd(a.dW2 + (size_t)r * kH + 16 * q + j, v[j]);
            tmem_ld16(c.tmem + c.lanef + kDW3 + 16 * q, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) atomicAdd(a.dW3 + (size_t)r * kH + 16 * q + j, v[j]);
        }
        if (c.part == 0) {
            tmem_ld16(c.tmem + c.lanef + kDW1, v);
#pragma unroll
            for (int j = 0; j < 3; ++j) atomicAdd(a.dW1 + (size_t)r * 3 + j, v[j]);
            atomicAdd(a.db1 + r, v[3]);
        } else if (c.part == 1) {
            tmem_ld16(c.tmem + c.lanef + kDW4, v);    // row r = h3 dim, column k = output k
#pragma unroll
            for (int k = 0; k < kS; ++k) atomicAdd(a.dW4 + (size_t)k * kH + r, v[k]);
        } else if (c.part == 2) {
            tmem_ld16(c.tmem + c.lanef + kDB2, v);
            atomicAdd(a.db2 + r, v[0]);
        } else {
            tmem_ld16(c.tmem + c.lanef + kDB3, v);
            atomicAdd(a.db3 + r, v[0]);
        }
        if (c.part == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
            if (lane == 0) atomicAdd(a.loss, lsum * a.scale);
            if ((lane & 1) == 0 && (lane >> 1) < kS) atomicAdd(a.db4 + (lane >> 1), db4acc);
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) tmem_dealloc(c.tmem, 512);
}

}  // namespace

// Reads and clears the smoothing kernel's timeout record.
le_status smooth_take_timeout(bool* timed_out)
{
    int flag = 0;
    LE_CUDA(cudaMemcpyFromSymbol(&flag, g_smooth_error, sizeof(int)));
    if (flag) {
        const int zero = 0;
        LE_CUDA(cudaMemcpyToSymbol(g_smooth_error, &zero, sizeof(int)));
    }
    *timed_out = flag != 0;
    return LE_OK;
}

}  // namespace leg

using namespace leg;

extern "C" le_status le_smooth(int32_t n, const float* means, const float* feat, const float* unc,
                               const le_smooth_mlp* mlp, float w_s, float lambda_smo, float* loss, float* d_feat,
                               int32_t d_feat_stride, const le_smooth_mlp_grads* dmlp, float* s_mlp, void* stream)
{
    LE_TRACE("le_smooth");
    LE_CHECK_ARG(n >= 0, "n = %d < 0", n);
    LE_CHECK_ARG(mlp && dmlp && loss, "null mlp / gradient / loss pointer");
    LE_CHECK_ARG(mlp->W1 && mlp->b1 && mlp->W2 && mlp->b2 && mlp->W3 && mlp->b3 && mlp->W4 && mlp->b4,
                 "null MLP parameter");
    LE_CHECK_ARG(dmlp->W1 && dmlp->b1 && dmlp->W2 && dmlp->b2 && dmlp->W3 && dmlp->b3 && dmlp->W4 && dmlp->b4,
                 "null MLP gradient");
    LE_CHECK_ARG(n == 0 || (means && feat && unc && d_feat), "null per-Gaussian pointer");
    LE_CHECK_ARG(d_feat_stride >= 8, "d_feat_stride = %d < 8", d_feat_stride);
    LE_CHECK_ARG(n == 0 || aligned16(feat), "feat must be 16-byte aligned");
    cudaStream_t s = as_stream(stream);
    LE_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), s));
    float* const gz[8] = {dmlp->W1, dmlp->b1, dmlp->W2, dmlp->b2, dmlp->W3, dmlp->b3, dmlp->W4, dmlp->b4};
    const size_t gn[8] = {kH * 3, kH, kH * kH, kH, kH * kH, kH, kS * kH, kS};
    for (int i = 0; i < 8; ++i) LE_CUDA(cudaMemsetAsync(gz[i], 0, gn[i] * sizeof(float), s));
    if (n == 0) return LE_OK;
    int dev = 0, sms = 0;
    LE_CUDA(cudaGetDevice(&dev));
    LE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SmoothArgs a;
    a.n = n;
    a.ntiles = (n + 127) / 128;
    a.means = means;
    a.feat = feat;
    a.unc = unc;
    a.W1 = mlp->W1;
    a.b1 = mlp->b1;
    a.W2 = mlp->W2;
    a.b2 = mlp->b2;
    a.W3 = mlp->W3;
    a.b3 = mlp->b3;
    a.W4 = mlp->W4;
    a.b4 = mlp->b4;
    a.w_s = w_s;
    a.scale = lambda_smo / (float)n;
    a.loss = loss;
    a.d_feat = d_feat;
    a.d_feat_stride = d_feat_stride;
    a.s_mlp = s_mlp;
    a.dW1 = dmlp->W1;
    a.db1 = dmlp->b1;
    a.dW2 = dmlp->W2;
    a.db2 = dmlp->b2;
    a.dW3 = dmlp->W3;
    a.db3 = dmlp->b3;
    a.dW4 = dmlp->W4;
    a.db4 = dmlp->b4;
    LE_CUDA(cudaFuncSetAttribute(smooth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmoothSmem));
    const int grid = a.ntiles < sms ? a.ntiles : sms;
    smooth_kernel<<<grid, kThreadsS, kSmoothSmem, s>>>(a);
    LE_LAUNCHED();
    return LE_OK;
}
