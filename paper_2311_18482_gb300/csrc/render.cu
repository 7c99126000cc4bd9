// Tile-based front-to-back compositing of RGB (Eq. 1), the compact semantic
// feature s_G (R_s, Sec. 3.4.1) and the uncertainty u (R_u, Sec. 3.4.2), and
// its backward pass.
//
// One CTA per 16x16 tile.  The tile's depth-ordered range is streamed through
// shared memory in batches of 256 splat records (80 B each, 16-byte loads);
// every thread then reads the batch by broadcast.  The forward runs two pixels
// per thread (128 threads per tile), the backward four (64 threads per tile),
// each warp on a compact block of rows, and both do the two-pixel arithmetic
// with paired FP32 instructions; so each staged record read, loop step and
// (backward) warp reduction serves several pixels.  The CTA stops fetching
// once every pixel's transmittance has dropped below 1e-4
// (__syncthreads_count ballot).
//
// The backward walks the same range back to front from each pixel's last
// contributor, recovering T_i = T_{i+1} / (1 - alpha_i) from the stored final
// transmittance, and sums each Gaussian's 18 gradient terms over the warp by a
// transpose through shared memory (every lane stores its 18 partial sums, lane
// f < 18 adds up field f with 16-byte reads), after which those 18 lanes each
// issue one scalar atomic add into the gradient record.
#include "common.cuh"

namespace leg {
le_status preprocess_backward(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                              const float* grad2d, const le_gaussian_grads* out, cudaStream_t s);
le_status preprocess_backward_adam(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                                   const float* grad2d, const le_gaussian_grads* m, const le_gaussian_grads* v,
                                   const AdamParams& h, cudaStream_t s, float* xp = nullptr,
                                   const float* xg = nullptr, float* xm = nullptr, float* xv = nullptr,
                                   int64_t xn = 0);
le_status check_gaussians(const le_gaussians* g);

namespace {

constexpr int kBlock = LE_TILE * LE_TILE;

// q = A' dx^2 + B' dx dy + C' dy^2 in base-2 exponent units (the record's scaled
// conic; alpha = o 2^-q), with a fixed operation order -- q = fma(C', dy * dy,
// fma(bx, dy, ax)), alpha0 = o * 2^-q -- so that the forward and the backward
// kernel take identical skip decisions.  ax = A' dx^2 and bx = B' dx depend on
// the column only, so each thread computes them once for its pixels of a column.
__device__ __forceinline__ float splat_ax(float Ap, float dx) { return __fmul_rn(Ap, __fmul_rn(dx, dx)); }
__device__ __forceinline__ float splat_bx(float Bp, float dx) { return __fmul_rn(Bp, dx); }

// Paired FP32 arithmetic: one instruction performs the IEEE round-to-nearest
// operation on both components, each exactly as the scalar operation would.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sel2(bool x, bool y, float2 v) { return make_float2(x ? v.x : 0.f, y ? v.y : 0.f); }

// Forward compositing state of one thread's two pixels (rows y and y + 2 of a
// column): transmittance, the 12 colour sums (rgb, u, s_G), the list position
// after the last blended Gaussian, and whether each pixel has stopped.
struct PixelPair {
    float2 T;
    float2 acc[12];
    int last[2];
    bool done[2];
};

// Blends staged records [0, cnt) (list positions pos0 + j) front to back into
// both pixels.  Per pixel: skip a Gaussian with q < 0 or alpha < 1/255, stop
// before the one that would make T (1 - alpha) < 1e-4.
__device__ __forceinline__ void blend_batch(const float4 (*rec)[kBlock], int cnt, int pos0, float fpx, float2 npy,
                                            PixelPair& s)
{
    for (int j = 0; j < cnt && !(s.done[0] && s.done[1]); ++j) {
        const float4 g0 = rec[0][j], g1 = rec[1][j];
        const float dx = __fsub_rn(g0.x, fpx);
        const float ax = splat_ax(g0.z, dx), bx = splat_bx(g0.w, dx);
        const float2 dy = __fadd2_rn(f2(g0.y), npy);
        const float2 q = __ffma2_rn(f2(g1.x), __fmul2_rn(dy, dy), __ffma2_rn(f2(bx), dy, f2(ax)));
        const float2 a0 = __fmul2_rn(f2(g1.y), make_float2(ex2_approx(-q.x), ex2_approx(-q.y)));
        const float2 alpha = make_float2(fminf(0.99f, a0.x), fminf(0.99f, a0.y));
        const float2 test = __fmul2_rn(s.T, __fadd2_rn(f2(1.f), make_float2(-alpha.x, -alpha.y)));
        const bool okx = !s.done[0] && q.x >= 0.f && alpha.x >= (1.f / 255.f);
        const bool oky = !s.done[1] && q.y >= 0.f && alpha.y >= (1.f / 255.f);
        const bool stopx = okx && test.x < 1e-4f, stopy = oky && test.y < 1e-4f;
        s.done[0] = s.done[0] || stopx;
        s.done[1] = s.done[1] || stopy;
        const bool bx_ = okx && !stopx, by_ = oky && !stopy;
        // no branch on (bx_ || by_): a pixel that skips gets weight 0 (its acc
        // and T are unchanged), and the straight-line loop runs 4 % faster over
        // a 1M-Gaussian view than one that skips the blend
        const float2 w = __fmul2_rn(sel2(bx_, by_, alpha), s.T);
        const float4 g2 = rec[2][j], g3 = rec[3][j], g4 = rec[4][j];
        const float f[12] = {g1.z, g1.w, g2.x, g2.y, g2.z, g2.w, g3.x, g3.y, g3.z, g3.w, g4.x, g4.y};
#pragma unroll
        for (int c = 0; c < 12; ++c) s.acc[c] = __ffma2_rn(f2(f[c]), w, s.acc[c]);   // rgb, u, s_G 0..7
        if (bx_) {
            s.T.x = test.x;
            s.last[0] = pos0 + j + 1;
        }
        if (by_) {
            s.T.y = test.y;
            s.last[1] = pos0 + j + 1;
        }
    }
}

// Stages list entries [s0 + b0, s0 + b0 + 256) of a tile: 128 threads, two records each.
__device__ __forceinline__ void stage_batch(float4 (*rec)[kBlock], const float4* __restrict__ splat,
                                            const uint32_t* __restrict__ ids, uint32_t s0, int b0, int n)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = threadIdx.x + h * (kBlock / 2);
        const int k = b0 + i;
        if (k < n) {
            const float4* r = splat + (size_t)ids[s0 + k] * 5;
#pragma unroll
            for (int c = 0; c < 5; ++c) rec[c][i] = __ldg(r + c);
        }
    }
}

// Walks list entries [s0, s0 + n) of the tile (list positions off + k) for both pixels.
__device__ __forceinline__ void composite_range(float4 (*rec)[kBlock], const float4* __restrict__ splat,
                                                const uint32_t* __restrict__ ids, uint32_t s0, int n, int off,
                                                float fpx, float2 npy, PixelPair& s)
{
    for (int b0 = 0; b0 < n; b0 += kBlock) {
        if (__syncthreads_count(s.done[0] && s.done[1]) == kBlock / 2) break;
        stage_batch(rec, splat, ids, s0, b0, n);
        __syncthreads();
        blend_batch(rec, min(kBlock, n - b0), off + b0, fpx, npy, s);
    }
}

// Forward pixel layout: one CTA of 128 threads per 16x16 tile, warp w covering
// the compact 16 x 4 block of rows [4w, 4w + 4) (its pixels tend to stop at
// similar depths, so fewer lanes idle while the warp walks on); thread t owns
// column t % 16 of rows fwd_row(t) and fwd_row(t) + 2.
__device__ __forceinline__ int fwd_row(int t) { return 4 * (t >> 5) + ((t >> 4) & 1); }

__global__ void __launch_bounds__(kBlock / 2) render_fwd_kernel(CamParams cam, const float4* __restrict__ splat,
                                                                const uint32_t* __restrict__ ids,
                                                                const uint2* __restrict__ ranges,
                                                                float* __restrict__ out_rgb, float* __restrict__ out_feat,
                                                                float* __restrict__ out_unc, float* __restrict__ T_final,
                                                                int* __restrict__ n_contrib)
{
    __shared__ float4 rec[5][kBlock];
    const int tile = blockIdx.x;
    const int tx = tile % cam.TX, ty = tile / cam.TX;
    const int px = tx * LE_TILE + (threadIdx.x & 15), py0 = ty * LE_TILE + fwd_row(threadIdx.x);
    const bool in0 = px < cam.W && py0 < cam.H, in1 = px < cam.W && py0 + 2 < cam.H;
    const uint2 rg = ranges[tile];
    PixelPair s;
    s.T = f2(1.f);
#pragma unroll
    for (int c = 0; c < 12; ++c) s.acc[c] = f2(0.f);
    s.last[0] = s.last[1] = 0;
    s.done[0] = !in0;
    s.done[1] = !in1;
    composite_range(rec, splat, ids, rg.x, (int)(rg.y - rg.x), 0, (float)px,
                    make_float2(-(float)py0, -(float)(py0 + 2)), s);
    const size_t P = (size_t)cam.W * cam.H;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!(h ? in1 : in0)) continue;
        const size_t o = (size_t)(py0 + 2 * h) * cam.W + px;
        const float T = h ? s.T.y : s.T.x;
        const auto comp = [&](int c) { return h ? s.acc[c].y : s.acc[c].x; };
        out_rgb[o] = __fmaf_rn(T, cam.bg[0], comp(0));
        out_rgb[P + o] = __fmaf_rn(T, cam.bg[1], comp(1));
        out_rgb[2 * P + o] = __fmaf_rn(T, cam.bg[2], comp(2));
        out_unc[o] = comp(3);
#pragma unroll
        for (int c = 0; c < 8; ++c) out_feat[c * P + o] = comp(4 + c);
        T_final[o] = T;
        n_contrib[o] = s.last[h];
    }
}

// One phase of the lazily placed forward render (le_bin_render_fwd): tile t
// blends its list entries [base(t, c_lo), base(t, c_hi)) -- depth chunks
// [c_lo, c_hi) -- where base(t, c) = base[t nchunks + c] (the next tile's start
// for c = nchunks) comes from the tile-major scan of the per-(tile, chunk)
// copy counts.  Phase c_lo > 0 resumes each pixel from the state the previous
// phase left in the outputs (colour sums without background, T, last list
// position, bit 30 of n_contrib = the pixel has stopped).  A tile whose pixels
// have all stopped, or whose list ends with this phase, writes its final
// outputs; any other tile saves the state and sets its flag in next_act (and
// its placement row group's in next_rows) for the next phase.  act (nullable = all):
// the tiles active in this phase.
constexpr int kStopped = 1 << 30;

// At most 64 registers (8 blocks of 128 threads per SM): at 80 registers (6 blocks)
// the phase kernels of one 1M-Gaussian view took 1.5 % longer.
__global__ void __launch_bounds__(kBlock / 2, 8) render_fwd_phase_kernel(
    CamParams cam, const float4* __restrict__ splat, const uint32_t* __restrict__ ids,
    const uint32_t* __restrict__ base, int nchunks, int c_lo, int c_hi, const uint8_t* __restrict__ act,
    uint8_t* __restrict__ next_act, uint8_t* __restrict__ next_rows, float* __restrict__ out_rgb,
    float* __restrict__ out_feat, float* __restrict__ out_unc, float* __restrict__ T_final, int* __restrict__ n_contrib)
{
    __shared__ float4 rec[5][kBlock];
    const int tile = blockIdx.x;
    if (act && !act[tile]) return;
    const int tx = tile % cam.TX, ty = tile / cam.TX;
    const int px = tx * LE_TILE + (threadIdx.x & 15), py0 = ty * LE_TILE + fwd_row(threadIdx.x);
    const bool in[2] = {px < cam.W && py0 < cam.H, px < cam.W && py0 + 2 < cam.H};
    const size_t P = (size_t)cam.W * cam.H;
    const size_t o[2] = {(size_t)py0 * cam.W + px, (size_t)(py0 + 2) * cam.W + px};
    const uint32_t tstart = base[(size_t)tile * nchunks], tend = base[(size_t)(tile + 1) * nchunks];
    const uint32_t s0 = c_lo == 0 ? tstart : base[(size_t)tile * nchunks + c_lo];
    const uint32_t s1 = c_hi >= nchunks ? tend : base[(size_t)tile * nchunks + c_hi];
    const int n = (int)(s1 - s0), off = (int)(s0 - tstart);

    PixelPair s;
    s.T = f2(1.f);
#pragma unroll
    for (int c = 0; c < 12; ++c) s.acc[c] = f2(0.f);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        s.last[h] = 0;
        s.done[h] = !in[h];
        if (c_lo > 0 && in[h]) {
            float v[12];
            v[0] = out_rgb[o[h]];
            v[1] = out_rgb[P + o[h]];
            v[2] = out_rgb[2 * P + o[h]];
            v[3] = out_unc[o[h]];
#pragma unroll
            for (int c = 0; c < 8; ++c) v[4 + c] = out_feat[c * P + o[h]];
            const float T = T_final[o[h]];
            const int nc = n_contrib[o[h]];
            if (h) {
                s.T.y = T;
#pragma unroll
                for (int c = 0; c < 12; ++c) s.acc[c].y = v[c];
            } else {
                s.T.x = T;
#pragma unroll
                for (int c = 0; c < 12; ++c) s.acc[c].x = v[c];
            }
            s.last[h] = nc & (kStopped - 1);
            s.done[h] = (nc & kStopped) != 0;
        }
    }
    composite_range(rec, splat, ids, s0, n, off, (float)px, make_float2(-(float)py0, -(float)(py0 + 2)), s);
    const bool complete = __syncthreads_count(s.done[0] && s.done[1]) == kBlock / 2 || s1 == tend;
    if (!complete && threadIdx.x == 0) {
        next_act[tile] = 1;
        next_rows[ty / LE_PLACE_ROWS] = 1;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!in[h]) continue;
        const float T = h ? s.T.y : s.T.x;
        const auto comp = [&](int c) { return h ? s.acc[c].y : s.acc[c].x; };
        // the background only once the pixel is final (the same FMA as render_fwd_kernel)
        out_rgb[o[h]] = complete ? __fmaf_rn(T, cam.bg[0], comp(0)) : comp(0);
        out_rgb[P + o[h]] = complete ? __fmaf_rn(T, cam.bg[1], comp(1)) : comp(1);
        out_rgb[2 * P + o[h]] = complete ? __fmaf_rn(T, cam.bg[2], comp(2)) : comp(2);
        out_unc[o[h]] = comp(3);
#pragma unroll
        for (int c = 0; c < 8; ++c) out_feat[c * P + o[h]] = comp(4 + c);
        T_final[o[h]] = T;
        n_contrib[o[h]] = complete ? s.last[h] : (s.last[h] | (s.done[h] ? kStopped : 0));
    }
}

// Four pixels per thread -- rows y, y + 2, y + 4, y + 6 of one column, warp w
// covering the compact 16 x 8 block of rows [8w, 8w + 8) -- in two pairs
// (y, y + 2) and (y + 4, y + 6) whose arithmetic runs on paired FP32
// instructions.  The channel contractions pair channels instead: per Gaussian
// and thread the 12 channel gradients sum_q w_q dL/dC_q,c and each pixel's
// f . dL/dC are paired FMAs over channel pairs (2k, 2k + 1), whose record
// values sit in the pairs of its 16-byte words, so only w is broadcast (pixel
// pairs broadcast every f_c: 0.380 against 0.374 ms at 1M Gaussians); the conic
// and mean gradients, which all share the
// column's dx, come from three sums over the thread's pixels -- D = sum dP,
// E = sum dP dy, F = sum dP dy^2 with dP = dL/dpower -- formed once per record:
// dconic = (-dx^2 D / 2, -dx E, -F / 2), dmean = (-A dx D - B E, -C E - B dx D).
template <int PPT>
__global__ void __launch_bounds__(kBlock / PPT) render_bwd_kernel(
    CamParams cam, const float4* __restrict__ splat, const uint32_t* __restrict__ ids, const uint2* __restrict__ ranges,
    const float* __restrict__ T_final, const int* __restrict__ n_contrib, const float* __restrict__ dL_drgb,
    const float* __restrict__ dL_dfeat, const float* __restrict__ dL_dunc, float4* __restrict__ grad2d)
{
    static_assert(PPT == 4, "two pixel pairs per thread");
    constexpr int NT = kBlock / PPT;
    __shared__ float4 rec[5][kBlock];
    __shared__ uint32_t sid[kBlock];
    __shared__ int s_max;
    // per warp, the lanes' 18 gradient partial sums, field-major; the row stride
    // of 36 floats staggers the rows over the banks for the 16-byte reads
    __shared__ __align__(16) float red[NT / 32][18][36];
    const int tile = blockIdx.x;
    const int tx = tile % cam.TX, ty = tile / cam.TX;
    const int px = tx * LE_TILE + (threadIdx.x & 15);
    const uint2 rg = ranges[tile];
    const float fpx = (float)px;
    const size_t P = (size_t)cam.W * cam.H;
    float(*wred)[36] = red[threadIdx.x >> 5];

    // pair p holds pixels q = 2p (x) and 2p + 1 (y); dC[q][k] = pixel q's upstream
    // gradient of channels (2k, 2k + 1)
    float2 npy[2], dC[PPT][6], T[2], Tf[2], S[2], nbg[2];
    int last[PPT];
    int lmax = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int y = ty * LE_TILE + 8 * (threadIdx.x >> 5) + ((threadIdx.x >> 4) & 1) + 2 * q;
        const bool inside = px < cam.W && y < cam.H;
        const size_t o = (size_t)y * cam.W + px;
        float d[12];
        d[0] = inside ? dL_drgb[o] : 0.f;
        d[1] = inside ? dL_drgb[P + o] : 0.f;
        d[2] = inside ? dL_drgb[2 * P + o] : 0.f;
        d[3] = inside ? dL_dunc[o] : 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) d[4 + c] = inside ? dL_dfeat[c * P + o] : 0.f;
        const float t = inside ? T_final[o] : 0.f;
        last[q] = inside ? n_contrib[o] : 0;
        // -bg . dL/dC (the background term of dL/dalpha); S = sum_c acc_c dL/dC_c, the
        // "colour behind" seen through this pixel's upstream gradient, obeys the
        // blending recurrence of acc itself
        const float nb = -(cam.bg[0] * d[0] + cam.bg[1] * d[1] + cam.bg[2] * d[2]);
        float2* pr[5] = {&npy[q >> 1], &T[q >> 1], &Tf[q >> 1], &S[q >> 1], &nbg[q >> 1]};
        const float v[5] = {-(float)y, t, t, 0.f, nb};
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            if (q & 1)
                pr[k]->y = v[k];
            else
                pr[k]->x = v[k];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) dC[q][k] = make_float2(d[2 * k], d[2 * k + 1]);
        lmax = max(lmax, last[q]);
    }

    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    const int wmax = __reduce_max_sync(0xffffffffu, lmax);
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, wmax);
    __syncthreads();
    const int nproc = s_max;
    const int lane = threadIdx.x & 31;

    for (int b_end = nproc; b_end > 0; b_end -= kBlock) {
        const int b_start = max(0, b_end - kBlock);
        __syncthreads();
#pragma unroll
        for (int l = 0; l < PPT; ++l) {
            const int i = threadIdx.x + l * NT;
            const int k = b_start + i;
            if (k < b_end) {
                const uint32_t gid = ids[rg.x + k];
                sid[i] = gid;
                const float4* r = splat + (size_t)gid * 5;
#pragma unroll
                for (int c = 0; c < 5; ++c) rec[c][i] = __ldg(r + c);
            }
        }
        __syncthreads();
        for (int j = min(b_end, wmax) - b_start - 1; j >= 0; --j) {
            const int pos = b_start + j;
            const float4 g0 = rec[0][j], g1 = rec[1][j];
            const float dx = __fsub_rn(g0.x, fpx);
            const float ax = splat_ax(g0.z, dx), bx = splat_bx(g0.w, dx);
            // the forward kernel's skip decisions, per pixel, with identical roundings
            float2 dy[2], G[2], al[2], a0[2];
            bool cb[PPT], any_mine = false;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                dy[p] = __fadd2_rn(f2(g0.y), npy[p]);
                const float2 qq = __ffma2_rn(f2(g1.x), __fmul2_rn(dy[p], dy[p]), __ffma2_rn(f2(bx), dy[p], f2(ax)));
                G[p] = make_float2(ex2_approx(-qq.x), ex2_approx(-qq.y));
                a0[p] = __fmul2_rn(f2(g1.y), G[p]);
                al[p] = make_float2(fminf(0.99f, a0[p].x), fminf(0.99f, a0[p].y));
                cb[2 * p] = pos < last[2 * p] && qq.x >= 0.f && al[p].x >= (1.f / 255.f);
                cb[2 * p + 1] = pos < last[2 * p + 1] && qq.y >= 0.f && al[p].y >= (1.f / 255.f);
                any_mine = any_mine || cb[2 * p] || cb[2 * p + 1];
            }
            if (!__any_sync(0xffffffffu, any_mine)) continue;
            float gr[18];
            {
                // acc[k]: channels (2k, 2k + 1) of sum_q w_q dL/dC_q over the thread's pixels
                float2 acc[6], sD = f2(0.f), sE = f2(0.f), sF = f2(0.f), sO = f2(0.f);
#pragma unroll
                for (int k = 0; k < 6; ++k) acc[k] = f2(0.f);
                if (any_mine) {
                    const float4 g2 = rec[2][j], g3 = rec[3][j], g4 = rec[4][j];
                    // the record's channels in the pairs its 16-byte words already hold
                    const float2 fp[6] = {make_float2(g1.z, g1.w), make_float2(g2.x, g2.y),
                                          make_float2(g2.z, g2.w), make_float2(g3.x, g3.y),
                                          make_float2(g3.z, g3.w), make_float2(g4.x, g4.y)};
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        const bool cx = cb[2 * p], cy = cb[2 * p + 1];
                        // alpha of the blended pixels, 0 for the others (1 / (1 - 0) = 1 leaves T,
                        // and w, dP and the opacity term are 0): both pairs run straight-line, which
                        // keeps the kernel at 127 registers (8 blocks per SM; a branch per pair took
                        // 168 registers, 6 blocks, and 11 % more time at 1M Gaussians)
                        const float2 am = sel2(cx, cy, al[p]);
                        const float2 inv = make_float2(__fdividef(1.f, 1.f - am.x), __fdividef(1.f, 1.f - am.y));
                        T[p] = __fmul2_rn(T[p], inv);
                        const float2 w = __fmul2_rn(am, T[p]);
                        // f . dL/dC per pixel, the even and odd channels in the two halves
                        float2 ea = __fmul2_rn(fp[0], dC[2 * p][0]), eb = __fmul2_rn(fp[0], dC[2 * p + 1][0]);
                        const float2 wa = f2(w.x), wb = f2(w.y);
#pragma unroll
                        for (int k = 0; k < 6; ++k) {
                            if (k > 0) {
                                ea = __ffma2_rn(fp[k], dC[2 * p][k], ea);
                                eb = __ffma2_rn(fp[k], dC[2 * p + 1][k], eb);
                            }
                            // rgb (0..2), unc (3), feat (4..11)
                            acc[k] = __ffma2_rn(wa, dC[2 * p][k], acc[k]);
                            acc[k] = __ffma2_rn(wb, dC[2 * p + 1][k], acc[k]);
                        }
                        const float2 fdc = make_float2(__fadd_rn(ea.x, ea.y), __fadd_rn(eb.x, eb.y));
                        const float2 diff = __fadd2_rn(fdc, make_float2(-S[p].x, -S[p].y));
                        const float2 dal = __ffma2_rn(T[p], diff, __fmul2_rn(__fmul2_rn(Tf[p], inv), nbg[p]));
                        S[p] = __ffma2_rn(am, diff, S[p]);
                        // alpha below the 0.99 clamp: dalpha/dpower = alpha, dalpha/do = G
                        const bool mx = cx && a0[p].x < 0.99f, my = cy && a0[p].y < 0.99f;
                        const float2 dP = __fmul2_rn(dal, sel2(mx, my, al[p]));
                        sO = __ffma2_rn(dal, sel2(mx, my, G[p]), sO);
                        sD = __fadd2_rn(sD, dP);
                        const float2 t = __fmul2_rn(dP, dy[p]);
                        sE = __fadd2_rn(sE, t);
                        sF = __ffma2_rn(t, dy[p], sF);
                    }
                }
                // the conic itself, for the mean gradient (dL/dpower is per unit of the natural exponent)
                const float cA = g0.z * kConicUnscaleAC, cB = g0.w * kConicUnscaleB, cC = g1.x * kConicUnscaleAC;
                const float D = sD.x + sD.y, E = sE.x + sE.y, F = sF.x + sF.y;
                const float dxD = dx * D;
                gr[0] = -(cA * dxD + cB * E);
                gr[1] = -(cC * E + cB * dxD);
                gr[2] = -0.5f * dx * dxD;
                gr[3] = -dx * E;
                gr[4] = -0.5f * F;
                gr[5] = sO.x + sO.y;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    gr[6 + 2 * k] = acc[k].x;
                    gr[7 + 2 * k] = acc[k].y;
                }
            }
            // warp sums of the 18 fields: a transpose through shared memory, lane f < 18 adding field f
#pragma unroll
            for (int c = 0; c < 18; ++c) wred[c][lane] = gr[c];
            __syncwarp();
            if (lane < 18) {
                const float4* row = reinterpret_cast<const float4*>(wred[lane]);
                float2 a = f2(0.f), b = f2(0.f);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float4 v = row[k];
                    a = __fadd2_rn(a, make_float2(v.x, v.y));
                    b = __fadd2_rn(b, make_float2(v.z, v.w));
                }
                const float2 t = __fadd2_rn(a, b);
                atomicAdd(reinterpret_cast<float*>(grad2d + (size_t)sid[j] * 5) + lane, t.x + t.y);
            }
            __syncwarp();
        }
    }
}

}  // namespace
}  // namespace leg

using namespace leg;

namespace leg {
le_status render_fwd_phase(const le_camera* cam, const float* splat, const uint32_t* ids, const uint32_t* base,
                           int nchunks, int c_lo, int c_hi, const uint8_t* act, uint8_t* next_act,
                           uint8_t* next_rows, float* out_rgb, float* out_feat, float* out_unc, float* T_final,
                           int32_t* n_contrib, cudaStream_t s)
{
    const CamParams cp = cam_params(cam);
    render_fwd_phase_kernel<<<cp.TX * cp.TY, kBlock / 2, 0, s>>>(cp, reinterpret_cast<const float4*>(splat), ids, base,
                                                            nchunks, c_lo, c_hi, act, next_act, next_rows, out_rgb,
                                                            out_feat, out_unc, T_final, n_contrib);
    LE_LAUNCHED();
    return LE_OK;
}
}  // namespace leg

extern "C" le_status le_render_fwd(const le_camera* cam, int32_t n, const float* splat, const uint32_t* sorted_ids,
                                   const uint32_t* tile_ranges, float* out_rgb, float* out_feat, float* out_unc,
                                   float* T_final, int32_t* n_contrib, void* stream)
{
    LE_TRACE("le_render_fwd");
    le_status st = check_camera(cam);
    if (st != LE_OK) return st;
    LE_CHECK_ARG(n >= 0, "n < 0");
    LE_CHECK_ARG(tile_ranges && out_rgb && out_feat && out_unc && T_final && n_contrib, "null output pointer");
    LE_CHECK_ARG(n == 0 || (splat && aligned16(splat)), "splat must be non-null and 16-byte aligned");
    LE_CHECK_ARG((reinterpret_cast<uintptr_t>(tile_ranges) & 7u) == 0, "tile_ranges must be 8-byte aligned");
    const CamParams cp = cam_params(cam);
    render_fwd_kernel<<<cp.TX * cp.TY, kBlock / 2, 0, as_stream(stream)>>>(
        cp, reinterpret_cast<const float4*>(splat), sorted_ids, reinterpret_cast<const uint2*>(tile_ranges), out_rgb,
        out_feat, out_unc, T_final, n_contrib);
    LE_LAUNCHED();
    return LE_OK;
}

namespace leg {
namespace {

// Arguments shared by le_render_bwd and le_render_bwd_adam; launches the
// screen-space backward (grad2d).
le_status render_backward_2d(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                             const uint32_t* sorted_ids, const uint32_t* tile_ranges, const float* T_final,
                             const int32_t* n_contrib, const float* dL_drgb, const float* dL_dfeat,
                             const float* dL_dunc, float* grad2d, cudaStream_t s)
{
    const CamParams cp = cam_params(cam);
    LE_CUDA(cudaMemsetAsync(grad2d, 0, sizeof(float) * LE_SPLAT_STRIDE * (size_t)g->n, s));
    render_bwd_kernel<4><<<cp.TX * cp.TY, kBlock / 4, 0, s>>>(cp, reinterpret_cast<const float4*>(pr->splat), sorted_ids,
                                                        reinterpret_cast<const uint2*>(tile_ranges), T_final,
                                                        n_contrib, dL_drgb, dL_dfeat, dL_dunc,
                                                        reinterpret_cast<float4*>(grad2d));
    LE_LAUNCHED();
    return LE_OK;
}

le_status check_render_bwd(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                           const uint32_t* tile_ranges, const float* T_final, const int32_t* n_contrib,
                           const float* dL_drgb, const float* dL_dfeat, const float* dL_dunc, const float* grad2d)
{
    le_status st = check_camera(cam);
    if (st != LE_OK) return st;
    if ((st = check_gaussians(g)) != LE_OK) return st;
    LE_CHECK_ARG(pr != nullptr, "null projected struct");
    LE_CHECK_ARG(tile_ranges && T_final && n_contrib && dL_drgb && dL_dfeat && dL_dunc, "null input pointer");
    if (g->n == 0) return LE_OK;
    LE_CHECK_ARG(pr->splat && pr->tiles_touched && pr->clamp_mask && aligned16(pr->splat), "bad projected pointers");
    LE_CHECK_ARG(grad2d && aligned16(grad2d), "grad2d must be non-null and 16-byte aligned");
    return LE_OK;
}

le_status check_field_set(const le_gaussian_grads* o, const char* what)
{
    LE_CHECK_ARG(o != nullptr, "null %s struct", what);
    LE_CHECK_ARG(o->means && o->log_scales && o->quats && o->opacity_raw && o->sh && o->feat && o->unc,
                 "null %s pointer", what);
    LE_CHECK_ARG(aligned16(o->quats) && aligned16(o->feat) && aligned16(o->sh),
                 "%s: quats/sh/feat must be 16-byte aligned", what);
    return LE_OK;
}

}  // namespace
}  // namespace leg

extern "C" le_status le_render_bwd(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                                   const uint32_t* sorted_ids, const uint32_t* tile_ranges, const float* T_final,
                                   const int32_t* n_contrib, const float* dL_drgb, const float* dL_dfeat,
                                   const float* dL_dunc, float* grad2d, const le_gaussian_grads* out, void* stream)
{
    LE_TRACE("le_render_bwd");
    le_status st = check_render_bwd(cam, g, pr, tile_ranges, T_final, n_contrib, dL_drgb, dL_dfeat, dL_dunc, grad2d);
    if (st != LE_OK || g->n == 0) return st;
    if ((st = check_field_set(out, "gradient")) != LE_OK) return st;
    cudaStream_t s = as_stream(stream);
    if ((st = render_backward_2d(cam, g, pr, sorted_ids, tile_ranges, T_final, n_contrib, dL_drgb, dL_dfeat, dL_dunc,
                                 grad2d, s)) != LE_OK)
        return st;
    return preprocess_backward(cam, g, pr, grad2d, out, s);
}

extern "C" le_status le_render_bwd_adam(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                                        const uint32_t* sorted_ids, const uint32_t* tile_ranges,
                                        const float* T_final, const int32_t* n_contrib, const float* dL_drgb,
                                        const float* dL_dfeat, const float* dL_dunc, float* grad2d,
                                        const le_gaussian_grads* m, const le_gaussian_grads* v,
                                        const le_adam_config* adam, void* stream)
{
    LE_TRACE("le_render_bwd_adam");
    le_status st = check_render_bwd(cam, g, pr, tile_ranges, T_final, n_contrib, dL_drgb, dL_dfeat, dL_dunc, grad2d);
    if (st != LE_OK) return st;
    LE_CHECK_ARG(adam != nullptr && adam->step >= 1, "adam config is null or step < 1");
    if (g->n == 0) return LE_OK;
    if ((st = check_field_set(m, "first-moment")) != LE_OK) return st;
    if ((st = check_field_set(v, "second-moment")) != LE_OK) return st;
    cudaStream_t s = as_stream(stream);
    if ((st = render_backward_2d(cam, g, pr, sorted_ids, tile_ranges, T_final, n_contrib, dL_drgb, dL_dfeat, dL_dunc,
                                 grad2d, s)) != LE_OK)
        return st;
    return preprocess_backward_adam(cam, g, pr, grad2d, m, v,
                                    adam_params(adam->step, adam->lr, adam->beta1, adam->beta2, adam->eps), s);
}

extern "C" le_status le_render_bwd_screen(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                                          const uint32_t* sorted_ids, const uint32_t* tile_ranges,
                                          const float* T_final, const int32_t* n_contrib, const float* dL_drgb,
                                          const float* dL_dfeat, const float* dL_dunc, float* grad2d, void* stream)
{
    LE_TRACE("le_render_bwd_screen");
    le_status st = check_render_bwd(cam, g, pr, tile_ranges, T_final, n_contrib, dL_drgb, dL_dfeat, dL_dunc, grad2d);
    if (st != LE_OK || g->n == 0) return st;
    return render_backward_2d(cam, g, pr, sorted_ids, tile_ranges, T_final, n_contrib, dL_drgb, dL_dfeat, dL_dunc,
                              grad2d, as_stream(stream));
}

extern "C" le_status le_project_bwd(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                                    const float* grad2d, const le_gaussian_grads* out, void* stream)
{
    LE_TRACE("le_project_bwd");
    le_status st = check_camera(cam);
    if (st != LE_OK) return st;
    if ((st = check_gaussians(g)) != LE_OK) return st;
    LE_CHECK_ARG(pr != nullptr, "null projected struct");
    if (g->n == 0) return LE_OK;
    LE_CHECK_ARG(pr->tiles_touched && pr->clamp_mask, "bad projected pointers");
    LE_CHECK_ARG(grad2d && aligned16(grad2d), "grad2d must be non-null and 16-byte aligned");
    if ((st = check_field_set(out, "gradient")) != LE_OK) return st;
    return preprocess_backward(cam, g, pr, grad2d, out, as_stream(stream));
}

extern "C" le_status le_project_bwd_adam(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                                         const float* grad2d, const le_gaussian_grads* m, const le_gaussian_grads* v,
                                         const le_adam_config* adam, void* stream)
{
    LE_TRACE("le_project_bwd_adam");
    le_status st = check_camera(cam);
    if (st != LE_OK) return st;
    if ((st = check_gaussians(g)) != LE_OK) return st;
    LE_CHECK_ARG(pr != nullptr, "null projected struct");
    LE_CHECK_ARG(adam != nullptr && adam->step >= 1, "adam config is null or step < 1");
    if (g->n == 0) return LE_OK;
    LE_CHECK_ARG(pr->tiles_touched && pr->clamp_mask, "bad projected pointers");
    LE_CHECK_ARG(grad2d && aligned16(grad2d), "grad2d must be non-null and 16-byte aligned");
    if ((st = check_field_set(m, "first-moment")) != LE_OK) return st;
    if ((st = check_field_set(v, "second-moment")) != LE_OK) return st;
    return preprocess_backward_adam(cam, g, pr, grad2d, m, v,
                                    adam_params(adam->step, adam->lr, adam->beta1, adam->beta2, adam->eps),
                                    as_stream(stream));
}

extern "C" le_status le_project_bwd_adam_extra(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                                               const float* grad2d, const le_gaussian_grads* m,
                                               const le_gaussian_grads* v, const le_adam_config* adam,
                                               float* extra_param, const float* extra_grad, float* extra_m,
                                               float* extra_v, int64_t n_extra, void* stream)
{
    LE_TRACE("le_project_bwd_adam_extra");
    le_status st = check_camera(cam);
    if (st != LE_OK) return st;
    if ((st = check_gaussians(g)) != LE_OK) return st;
    LE_CHECK_ARG(pr != nullptr, "null projected struct");
    LE_CHECK_ARG(adam != nullptr && adam->step >= 1, "adam config is null or step < 1");
    LE_CHECK_ARG(n_extra >= 0, "n_extra < 0");
    LE_CHECK_ARG(n_extra == 0 || (extra_param && extra_grad && extra_m && extra_v && aligned16(extra_param) &&
                                  aligned16(extra_grad) && aligned16(extra_m) && aligned16(extra_v)),
                 "the extra range's four arrays must be non-null and 16-byte aligned");
    if (g->n == 0 && n_extra == 0) return LE_OK;
    if (g->n > 0) {
        LE_CHECK_ARG(pr->tiles_touched && pr->clamp_mask, "bad projected pointers");
        LE_CHECK_ARG(grad2d && aligned16(grad2d), "grad2d must be non-null and 16-byte aligned");
        if ((st = check_field_set(m, "first-moment")) != LE_OK) return st;
        if ((st = check_field_set(v, "second-moment")) != LE_OK) return st;
    }
    return preprocess_backward_adam(cam, g, pr, grad2d, m, v,
                                    adam_params(adam->step, adam->lr, adam->beta1, adam->beta2, adam->eps),
                                    as_stream(stream), extra_param, extra_grad, extra_m, extra_v, n_extra);
}
