// Tile-based front-to-back compositing of RGB (Eq. 1), the compact semantic
// feature s_G (R_s, Sec. 3.4.1) and the uncertainty u (R_u, Sec. 3.4.2), and
// its backward pass.
//
// One CTA per 16x16 tile.  The tile's depth-ordered range is streamed through
// shared memory in batches of 256 splat records (80 B each, 16-byte loads);
// every thread then reads the batch by broadcast.  The forward runs one pixel
// per thread (pixels stop at different depths; pairing them costs more than it
// saves), the backward four (rows y, y + 4, y + 8, y + 12; 64 threads per
// tile), so each staged record read, each loop step and each warp reduction
// serves four pixels.  The CTA stops fetching once every pixel's
// transmittance has dropped below 1e-4 (__syncthreads_count ballot).
//
// The backward walks the same range back to front from each pixel's last
// contributor, recovering T_i = T_{i+1} / (1 - alpha_i) from the stored final
// transmittance, sums each Gaussian's 18 gradient terms over the warp with a
// recursive-halving shuffle reduction (20 shuffles instead of 18 x 5) after
// which 18 lanes each issue one scalar atomic add into the gradient record.
#include "common.cuh"

namespace leg {
le_status preprocess_backward(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                              const float* grad2d, const le_gaussian_grads* out, cudaStream_t s);
le_status preprocess_backward_adam(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                                   const float* grad2d, const le_gaussian_grads* m, const le_gaussian_grads* v,
                                   const AdamParams& h, cudaStream_t s);
le_status check_gaussians(const le_gaussians* g);

namespace {

constexpr int kBlock = LE_TILE * LE_TILE;

// q = A' dx^2 + B' dx dy + C' dy^2 in base-2 exponent units (the record's scaled
// conic; alpha = o 2^-q), with a fixed operation order: the forward and the
// backward kernel take identical skip decisions.  ax = A' dx^2 and bx = B' dx
// depend on the column only, so the backward computes them once for its two
// pixels of a column.
__device__ __forceinline__ float splat_ax(float Ap, float dx) { return __fmul_rn(Ap, __fmul_rn(dx, dx)); }
__device__ __forceinline__ float splat_bx(float Bp, float dx) { return __fmul_rn(Bp, dx); }
__device__ __forceinline__ float splat_q(float ax, float bx, float Cp, float dy)
{
    return __fmaf_rn(Cp, __fmul_rn(dy, dy), __fmaf_rn(bx, dy, ax));
}

__device__ __forceinline__ float splat_alpha0(float opacity, float q)
{
    return __fmul_rn(opacity, ex2_approx(-q));
}

__global__ void __launch_bounds__(kBlock) render_fwd_kernel(CamParams cam, const float4* __restrict__ splat,
                                                            const uint32_t* __restrict__ ids,
                                                            const uint2* __restrict__ ranges,
                                                            float* __restrict__ out_rgb, float* __restrict__ out_feat,
                                                            float* __restrict__ out_unc, float* __restrict__ T_final,
                                                            int* __restrict__ n_contrib)
{
    __shared__ float4 rec[5][kBlock];
    const int tile = blockIdx.x;
    const int tx = tile % cam.TX, ty = tile / cam.TX;
    const int px = tx * LE_TILE + (threadIdx.x & 15), py = ty * LE_TILE + (threadIdx.x >> 4);
    const bool inside = px < cam.W && py < cam.H;
    const uint2 rg = ranges[tile];
    const int n = (int)(rg.y - rg.x);
    const float fpx = (float)px, fpy = (float)py;

    bool done = !inside;
    float T = 1.f;
    float acc[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = 0.f;
    int last = 0;

    for (int b0 = 0; b0 < n; b0 += kBlock) {
        if (__syncthreads_count(done) == kBlock) break;
        const int k = b0 + threadIdx.x;
        if (k < n) {
            const float4* r = splat + (size_t)ids[rg.x + k] * 5;
#pragma unroll
            for (int q = 0; q < 5; ++q) rec[q][threadIdx.x] = __ldg(r + q);
        }
        __syncthreads();
        const int cnt = min(kBlock, n - b0);
        for (int j = 0; !done && j < cnt; ++j) {
            const float4 g0 = rec[0][j], g1 = rec[1][j];
            const float dx = __fsub_rn(g0.x, fpx), dy = __fsub_rn(g0.y, fpy);
            const float q = splat_q(splat_ax(g0.z, dx), splat_bx(g0.w, dx), g1.x, dy);
            if (q < 0.f) continue;
            const float alpha = fminf(0.99f, splat_alpha0(g1.y, q));
            if (alpha < (1.f / 255.f)) continue;
            const float test = T * (1.f - alpha);
            if (test < 1e-4f) {
                done = true;
                break;
            }
            const float w = alpha * T;
            const float4 g2 = rec[2][j], g3 = rec[3][j], g4 = rec[4][j];
            acc[0] = fmaf(g1.z, w, acc[0]);
            acc[1] = fmaf(g1.w, w, acc[1]);
            acc[2] = fmaf(g2.x, w, acc[2]);
            acc[3] = fmaf(g2.y, w, acc[3]);     // uncertainty
            acc[4] = fmaf(g2.z, w, acc[4]);     // feature 0..7
            acc[5] = fmaf(g2.w, w, acc[5]);
            acc[6] = fmaf(g3.x, w, acc[6]);
            acc[7] = fmaf(g3.y, w, acc[7]);
            acc[8] = fmaf(g3.z, w, acc[8]);
            acc[9] = fmaf(g3.w, w, acc[9]);
            acc[10] = fmaf(g4.x, w, acc[10]);
            acc[11] = fmaf(g4.y, w, acc[11]);
            T = test;
            last = b0 + j + 1;
        }
    }
    if (!inside) return;
    const size_t P = (size_t)cam.W * cam.H, o = (size_t)py * cam.W + px;
    out_rgb[o] = __fmaf_rn(T, cam.bg[0], acc[0]);
    out_rgb[P + o] = __fmaf_rn(T, cam.bg[1], acc[1]);
    out_rgb[2 * P + o] = __fmaf_rn(T, cam.bg[2], acc[2]);
    out_unc[o] = acc[3];
#pragma unroll
    for (int c = 0; c < 8; ++c) out_feat[c * P + o] = acc[4 + c];
    T_final[o] = T;
    n_contrib[o] = last;
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

__global__ void __launch_bounds__(kBlock) render_fwd_phase_kernel(
    CamParams cam, const float4* __restrict__ splat, const uint32_t* __restrict__ ids,
    const uint32_t* __restrict__ base, int nchunks, int c_lo, int c_hi, const uint8_t* __restrict__ act,
    uint8_t* __restrict__ next_act, uint8_t* __restrict__ next_rows, float* __restrict__ out_rgb,
    float* __restrict__ out_feat, float* __restrict__ out_unc, float* __restrict__ T_final, int* __restrict__ n_contrib)
{
    __shared__ float4 rec[5][kBlock];
    const int tile = blockIdx.x;
    if (act && !act[tile]) return;
    const int tx = tile % cam.TX, ty = tile / cam.TX;
    const int px = tx * LE_TILE + (threadIdx.x & 15), py = ty * LE_TILE + (threadIdx.x >> 4);
    const bool inside = px < cam.W && py < cam.H;
    const size_t P = (size_t)cam.W * cam.H, o = (size_t)py * cam.W + px;
    const uint32_t tstart = base[(size_t)tile * nchunks], tend = base[(size_t)(tile + 1) * nchunks];
    const uint32_t s0 = c_lo == 0 ? tstart : base[(size_t)tile * nchunks + c_lo];
    const uint32_t s1 = c_hi >= nchunks ? tend : base[(size_t)tile * nchunks + c_hi];
    const int n = (int)(s1 - s0), off = (int)(s0 - tstart);
    const float fpx = (float)px, fpy = (float)py;

    bool done = !inside;
    float T = 1.f;
    float acc[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = 0.f;
    int last = 0;
    if (c_lo > 0 && inside) {
        T = T_final[o];
        acc[0] = out_rgb[o];
        acc[1] = out_rgb[P + o];
        acc[2] = out_rgb[2 * P + o];
        acc[3] = out_unc[o];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[4 + c] = out_feat[c * P + o];
        const int nc = n_contrib[o];
        last = nc & (kStopped - 1);
        done = (nc & kStopped) != 0;
    }

    for (int b0 = 0; b0 < n; b0 += kBlock) {
        if (__syncthreads_count(done) == kBlock) break;
        const int k = b0 + threadIdx.x;
        if (k < n) {
            const float4* r = splat + (size_t)ids[s0 + k] * 5;
#pragma unroll
            for (int q = 0; q < 5; ++q) rec[q][threadIdx.x] = __ldg(r + q);
        }
        __syncthreads();
        const int cnt = min(kBlock, n - b0);
        for (int j = 0; !done && j < cnt; ++j) {
            const float4 g0 = rec[0][j], g1 = rec[1][j];
            const float dx = __fsub_rn(g0.x, fpx), dy = __fsub_rn(g0.y, fpy);
            const float q = splat_q(splat_ax(g0.z, dx), splat_bx(g0.w, dx), g1.x, dy);
            if (q < 0.f) continue;
            const float alpha = fminf(0.99f, splat_alpha0(g1.y, q));
            if (alpha < (1.f / 255.f)) continue;
            const float test = T * (1.f - alpha);
            if (test < 1e-4f) {
                done = true;
                break;
            }
            const float w = alpha * T;
            const float4 g2 = rec[2][j], g3 = rec[3][j], g4 = rec[4][j];
            acc[0] = fmaf(g1.z, w, acc[0]);
            acc[1] = fmaf(g1.w, w, acc[1]);
            acc[2] = fmaf(g2.x, w, acc[2]);
            acc[3] = fmaf(g2.y, w, acc[3]);
            acc[4] = fmaf(g2.z, w, acc[4]);
            acc[5] = fmaf(g2.w, w, acc[5]);
            acc[6] = fmaf(g3.x, w, acc[6]);
            acc[7] = fmaf(g3.y, w, acc[7]);
            acc[8] = fmaf(g3.z, w, acc[8]);
            acc[9] = fmaf(g3.w, w, acc[9]);
            acc[10] = fmaf(g4.x, w, acc[10]);
            acc[11] = fmaf(g4.y, w, acc[11]);
            T = test;
            last = off + b0 + j + 1;
        }
    }
    const bool complete = __syncthreads_count(done) == kBlock || s1 == tend;
    if (!complete && threadIdx.x == 0) {
        next_act[tile] = 1;
        next_rows[ty / LE_PLACE_ROWS] = 1;
    }
    if (!inside) return;
    // the background only once the pixel is final (the same FMA as render_fwd_kernel)
    out_rgb[o] = complete ? __fmaf_rn(T, cam.bg[0], acc[0]) : acc[0];
    out_rgb[P + o] = complete ? __fmaf_rn(T, cam.bg[1], acc[1]) : acc[1];
    out_rgb[2 * P + o] = complete ? __fmaf_rn(T, cam.bg[2], acc[2]) : acc[2];
    out_unc[o] = acc[3];
#pragma unroll
    for (int c = 0; c < 8; ++c) out_feat[c * P + o] = acc[4 + c];
    T_final[o] = T;
    n_contrib[o] = complete ? last : (last | (done ? kStopped : 0));
}

// One stage of a recursive-halving ("transpose") reduction of N values held by
// every lane: lanes with bit O set keep the upper half of the values, the
// others the lower half, each adding its partner's copy of the half it keeps.
template <int N, int O>
__device__ __forceinline__ void halve(float* v, bool upper)
{
    constexpr int H = (N + 1) / 2;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const float lo = v[i];
        const float hi = (i + H < N) ? v[i + H] : 0.f;
        const float recv = __shfl_xor_sync(0xffffffffu, upper ? lo : hi, O);
        v[i] = (upper ? hi : lo) + recv;
    }
}

// Warp-wide sums of 18 values in 9+5+3+2+1 = 20 shuffles; afterwards v[0] of
// lane l is the sum of value field_of_lane(l) (or nothing, when that is -1).
__device__ __forceinline__ void warp_sum18(float* v, int lane)
{
    halve<18, 16>(v, lane & 16);
    halve<9, 8>(v, lane & 8);
    halve<5, 4>(v, lane & 4);
    halve<3, 2>(v, lane & 2);
    halve<2, 1>(v, lane & 1);
}

__device__ __forceinline__ int field_of_lane(int lane)
{
    int valid = 18, base = 0;
    const int H[5] = {9, 5, 3, 2, 1}, O[5] = {16, 8, 4, 2, 1};
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        if (lane & O[s]) {
            base += H[s];
            valid = valid > H[s] ? valid - H[s] : 0;
        } else {
            valid = valid < H[s] ? valid : H[s];
        }
    }
    return valid >= 1 ? base : -1;
}

template <int PPT>
__global__ void __launch_bounds__(kBlock / PPT) render_bwd_kernel(
    CamParams cam, const float4* __restrict__ splat, const uint32_t* __restrict__ ids, const uint2* __restrict__ ranges,
    const float* __restrict__ T_final, const int* __restrict__ n_contrib, const float* __restrict__ dL_drgb,
    const float* __restrict__ dL_dfeat, const float* __restrict__ dL_dunc, float4* __restrict__ grad2d)
{
    constexpr int NT = kBlock / PPT;
    __shared__ float4 rec[5][kBlock];
    __shared__ uint32_t sid[kBlock];
    __shared__ int s_max;
    const int tile = blockIdx.x;
    const int tx = tile % cam.TX, ty = tile / cam.TX;
    const int px = tx * LE_TILE + (threadIdx.x & 15);
    const uint2 rg = ranges[tile];
    const float fpx = (float)px;
    const size_t P = (size_t)cam.W * cam.H;

    float py[PPT], dC[PPT][12], T[PPT], Tf[PPT], S[PPT], bgdot[PPT];
    int last[PPT];
    int lmax = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const int y = ty * LE_TILE + (threadIdx.x >> 4) + q * (LE_TILE / PPT);
        py[q] = (float)y;
        const bool inside = px < cam.W && y < cam.H;
        const size_t o = (size_t)y * cam.W + px;
        T[q] = inside ? T_final[o] : 0.f;
        last[q] = inside ? n_contrib[o] : 0;
        dC[q][0] = inside ? dL_drgb[o] : 0.f;
        dC[q][1] = inside ? dL_drgb[P + o] : 0.f;
        dC[q][2] = inside ? dL_drgb[2 * P + o] : 0.f;
        dC[q][3] = inside ? dL_dunc[o] : 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) dC[q][4 + c] = inside ? dL_dfeat[c * P + o] : 0.f;
        Tf[q] = T[q];
        // S = sum_c acc_c dL/dC_c, the "colour behind" seen through this pixel's
        // upstream gradient; it obeys the blending recurrence of acc itself.
        S[q] = 0.f;
        bgdot[q] = cam.bg[0] * dC[q][0] + cam.bg[1] * dC[q][1] + cam.bg[2] * dC[q][2];
        lmax = max(lmax, last[q]);
    }

    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    const int wmax = __reduce_max_sync(0xffffffffu, lmax);
    if ((threadIdx.x & 31) == 0) atomicMax(&s_max, wmax);
    __syncthreads();
    const int nproc = s_max;
    const int lane = threadIdx.x & 31;
    const int my_field = field_of_lane(lane);

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
            float dy[PPT], G[PPT], a0[PPT], alpha[PPT];
            bool contrib[PPT], any_mine = false;
#pragma unroll
            for (int q = 0; q < PPT; ++q) {
                dy[q] = __fsub_rn(g0.y, py[q]);
                const float qq = splat_q(ax, bx, g1.x, dy[q]);
                G[q] = ex2_approx(-qq);
                a0[q] = __fmul_rn(g1.y, G[q]);
                alpha[q] = fminf(0.99f, a0[q]);
                contrib[q] = pos < last[q] && qq >= 0.f && alpha[q] >= (1.f / 255.f);
                any_mine = any_mine || contrib[q];
            }
            if (!__any_sync(0xffffffffu, any_mine)) continue;
            float gr[18];
#pragma unroll
            for (int c = 0; c < 18; ++c) gr[c] = 0.f;
            if (any_mine) {
                const float4 g2 = rec[2][j], g3 = rec[3][j], g4 = rec[4][j];
                // the conic itself, for the mean gradient (dL/dpower is per unit of the natural exponent)
                const float cA = g0.z * kConicUnscaleAC, cB = g0.w * kConicUnscaleB, cC = g1.x * kConicUnscaleAC;
                const float f[12] = {g1.z, g1.w, g2.x, g2.y, g2.z, g2.w, g3.x, g3.y, g3.z, g3.w, g4.x, g4.y};
#pragma unroll
                for (int q = 0; q < PPT; ++q) {
                    if (!contrib[q]) continue;
                    const float inv1ma = __fdividef(1.f, 1.f - alpha[q]);
                    T[q] *= inv1ma;
                    const float w = alpha[q] * T[q];
                    float fdc = 0.f;
#pragma unroll
                    for (int c = 0; c < 12; ++c) {
                        gr[6 + c] = fmaf(w, dC[q][c], gr[6 + c]);      // rgb (6..8), unc (9), feat (10..17)
                        fdc = fmaf(f[c], dC[q][c], fdc);
                    }
                    const float dalpha = T[q] * (fdc - S[q]) - Tf[q] * inv1ma * bgdot[q];
                    S[q] = fmaf(alpha[q], fdc - S[q], S[q]);
                    if (a0[q] < 0.99f) {
                        const float dpow = dalpha * alpha[q];
                        gr[5] = fmaf(dalpha, G[q], gr[5]);
                        gr[2] = fmaf(-0.5f * dpow * dx, dx, gr[2]);
                        gr[3] = fmaf(-dpow * dx, dy[q], gr[3]);
                        gr[4] = fmaf(-0.5f * dpow * dy[q], dy[q], gr[4]);
                        gr[0] = fmaf(dpow, -cA * dx - cB * dy[q], gr[0]);
                        gr[1] = fmaf(dpow, -cC * dy[q] - cB * dx, gr[1]);
                    }
                }
            }
            warp_sum18(gr, lane);
            if (my_field >= 0) atomicAdd(reinterpret_cast<float*>(grad2d + (size_t)sid[j] * 5) + my_field, gr[0]);
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
    render_fwd_phase_kernel<<<cp.TX * cp.TY, kBlock, 0, s>>>(cp, reinterpret_cast<const float4*>(splat), ids, base,
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
    render_fwd_kernel<<<cp.TX * cp.TY, kBlock, 0, as_stream(stream)>>>(
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
