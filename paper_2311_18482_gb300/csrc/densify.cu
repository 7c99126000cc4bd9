// Adaptive density control of 3D Gaussian Splatting, which Sec. 4 keeps
// (clone / split / prune, opacity reset), as the steps the training loop calls:
//   le_densify_stats  every step: acc_i += |dL/dmean2d_i| (pixels), cnt_i += 1
//                     and max_radius_i = max(max_radius_i, radius_i) for every
//                     Gaussian with a nonzero screen radius;
//   le_opacity_reset  every few thousand steps: opacity = min(opacity, 0.01),
//                     the opacity's Adam moments zeroed;
//   le_densify        every few hundred steps: classify each Gaussian (pruned,
//                     kept, kept + clone, split), count the three output
//                     segments per block, scan the block counts, then scatter
//                     parameters and Adam moments into the caller's output
//                     arrays: kept and cloned Gaussians (index order), clones
//                     (index order), two children per split Gaussian.
// The decisions use FP32 comparisons against thresholds derived once in double
// (no transcendental function on the device), so they are reproducible bit for
// bit: opacity_raw < logit(min_opacity); max log-scale > ln(percent_dense *
// extent); cnt > 0 and acc >= fl(grad_thresh * cnt); and, when enabled, the
// size tests that prune Gaussians too large on screen (max_radius >
// max_screen_size) or in the world (max log-scale > ln(world_frac * extent)).  A split child k copies
// its parent except mean = mu + R(q) diag(exp(log-scale)) n_k (the caller's
// standard normal samples) and log-scale - ln(1.6); clones and children start
// with zero Adam moments.
#include "common.cuh"

namespace leg {
namespace {

constexpr int kDB = 1024;                  // Gaussians per classification block

struct DensifyThresholds {
    float grad_thresh, log_big, logit_min, ln16, max_screen, log_world;
};

struct Fields {
    float* f[7];
};

__host__ __device__ constexpr int field_w(int f, int nc)
{
    return f == 4 ? 3 * nc : (f == 2 ? 4 : (f == 5 ? 8 : (f <= 1 ? 3 : 1)));
}

__global__ void densify_stats_kernel(int n, const float4* __restrict__ grad2d, const int* __restrict__ radius,
                                     float* __restrict__ acc, int* __restrict__ cnt, int* __restrict__ max_radius)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = radius[i];
    if (r <= 0) return;
    const float4 g = grad2d[5 * (size_t)i];
    acc[i] = __fadd_rn(acc[i], __fsqrt_rn(__fadd_rn(__fmul_rn(g.x, g.x), __fmul_rn(g.y, g.y))));
    cnt[i] += 1;
    if (max_radius && r > max_radius[i]) max_radius[i] = r;
}

// opacity_raw = min(opacity_raw, logit_max); the opacity's Adam moments zeroed.
__global__ void opacity_reset_kernel(int n, float* __restrict__ op, float* __restrict__ m, float* __restrict__ v,
                                     float logit_max)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    op[i] = fminf(op[i], logit_max);
    m[i] = 0.f;
    v[i] = 0.f;
}

__device__ __forceinline__ int classify(int i, const float* ls, const float* op, const float* acc, const int* cnt,
                                        const int* max_radius, const DensifyThresholds& t)
{
    const float smax = fmaxf(fmaxf(ls[3 * i], ls[3 * i + 1]), ls[3 * i + 2]);
    const int c = cnt[i];
    const bool cand = c > 0 && acc[i] >= __fmul_rn(t.grad_thresh, (float)c);
    const bool big_screen = t.max_screen > 0.f && (float)max_radius[i] > t.max_screen;
    if (op[i] < t.logit_min || big_screen || smax > t.log_world) return 0;
    if (cand) return smax > t.log_big ? 3 : 2;
    return 1;
}

// kind[i] and per-block counts of the three output segments: [3][nblocks].
__global__ void __launch_bounds__(256) densify_count_kernel(int n, const float* __restrict__ ls,
                                                            const float* __restrict__ op, const float* __restrict__ acc,
                                                            const int* __restrict__ cnt,
                                                            const int* __restrict__ max_radius, DensifyThresholds t,
                                                            uint8_t* __restrict__ kind, unsigned* __restrict__ bcount)
{
    __shared__ unsigned c3[3];
    if (threadIdx.x < 3) c3[threadIdx.x] = 0;
    __syncthreads();
    unsigned k1 = 0, k2 = 0, k3 = 0;
    for (int r = 0; r < kDB / 256; ++r) {
        const int i = blockIdx.x * kDB + r * 256 + threadIdx.x;
        if (i < n) {
            const int k = classify(i, ls, op, acc, cnt, max_radius, t);
            kind[i] = (uint8_t)k;
            k1 += k == 1 || k == 2;
            k2 += k == 2;
            k3 += k == 3;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        k1 += __shfl_xor_sync(0xffffffffu, k1, o);
        k2 += __shfl_xor_sync(0xffffffffu, k2, o);
        k3 += __shfl_xor_sync(0xffffffffu, k3, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&c3[0], k1);
        atomicAdd(&c3[1], k2);
        atomicAdd(&c3[2], k3);
    }
    __syncthreads();
    if (threadIdx.x < 3) bcount[threadIdx.x * gridDim.x + blockIdx.x] = c3[threadIdx.x];
}

// Exclusive scan of each segment's block counts, in place; totals[3].  One block.
__global__ void __launch_bounds__(1024) densify_scan_kernel(unsigned* bcount, int nb, unsigned long long* totals)
{
    __shared__ unsigned long long carry;
    __shared__ unsigned wsum[32];
    for (int sgm = 0; sgm < 3; ++sgm) {
        unsigned* c = bcount + (size_t)sgm * nb;
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (int b0 = 0; b0 < nb; b0 += 1024) {
            const int b = b0 + threadIdx.x;
            const unsigned v = b < nb ? c[b] : 0u;
            unsigned x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if ((threadIdx.x & 31) >= o) x += y;
            }
            if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
            __syncthreads();
            if (threadIdx.x < 32) {
                unsigned w = wsum[threadIdx.x];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(0xffffffffu, w, o);
                    if (threadIdx.x >= o) w += y;
                }
                wsum[threadIdx.x] = w;
            }
            __syncthreads();
            const unsigned incl = x + ((threadIdx.x >> 5) > 0 ? wsum[(threadIdx.x >> 5) - 1] : 0u);
            if (b < nb) c[b] = (unsigned)(carry + incl - v);
            __syncthreads();
            if (threadIdx.x == 1023) carry += incl;
            __syncthreads();
        }
        if (threadIdx.x == 0) totals[sgm] = carry;
        __syncthreads();
    }
}

struct ScatterArgs {
    int n, nc;
    Fields p, m, v;                 // inputs
    Fields po, mo, vo;              // outputs
    const uint8_t* kind;
    const unsigned* boff;           // [3][nblocks] exclusive block offsets
    const unsigned long long* totals;
    const float* noise;             // [n][2][3]
    float ln16;
};

// Copies Gaussian src to output slot dst in every field (moments or zeros);
// 16-byte accesses for the fields whose rows are whole multiples of 16 bytes
// (quaternions, SH, features) when the arrays allow it, scalar ones otherwise.
__device__ __forceinline__ void copy_gaussian(const ScatterArgs& a, size_t src, size_t dst, bool moments)
{
#pragma unroll
    for (int f = 0; f < 7; ++f) {
        const int w = field_w(f, a.nc);
        const float* ps = a.p.f[f];
        const float* ms = a.m.f[f];
        const float* vs = a.v.f[f];
        float* pd = a.po.f[f];
        float* md = a.mo.f[f];
        float* vd = a.vo.f[f];
        if ((w & 3) == 0 && ((reinterpret_cast<uintptr_t>(ps) | reinterpret_cast<uintptr_t>(ms) |
                              reinterpret_cast<uintptr_t>(vs) | reinterpret_cast<uintptr_t>(pd) |
                              reinterpret_cast<uintptr_t>(md) | reinterpret_cast<uintptr_t>(vd)) & 15u) == 0) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int e = 0; e < w; e += 4) {
                reinterpret_cast<float4*>(pd + dst * w)[e >> 2] = reinterpret_cast<const float4*>(ps + src * w)[e >> 2];
                reinterpret_cast<float4*>(md + dst * w)[e >> 2] =
                    moments ? reinterpret_cast<const float4*>(ms + src * w)[e >> 2] : z;
                reinterpret_cast<float4*>(vd + dst * w)[e >> 2] =
                    moments ? reinterpret_cast<const float4*>(vs + src * w)[e >> 2] : z;
            }
        } else {
            for (int e = 0; e < w; ++e) {
                pd[dst * w + e] = ps[src * w + e];
                md[dst * w + e] = moments ? ms[src * w + e] : 0.f;
                vd[dst * w + e] = moments ? vs[src * w + e] : 0.f;
            }
        }
    }
}

// Positions: block offset + rank within the block (a block-wide scan of the
// three flags, in index order), then the copies.
__global__ void __launch_bounds__(256) densify_scatter_kernel(ScatterArgs a)
{
    __shared__ unsigned wsum[3][8];
    __shared__ unsigned run[3];
    if (threadIdx.x < 3) run[threadIdx.x] = 0;
    __syncthreads();
    const int nb = gridDim.x;
    const unsigned long long K1 = a.totals[0], K2 = a.totals[1];
    for (int r = 0; r < kDB / 256; ++r) {
        const int i = blockIdx.x * kDB + r * 256 + threadIdx.x;
        const int k = i < a.n ? a.kind[i] : 0;
        const unsigned f[3] = {(unsigned)(k == 1 || k == 2), (unsigned)(k == 2), (unsigned)(k == 3)};
        unsigned ex[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            unsigned x = f[s];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if ((threadIdx.x & 31) >= o) x += y;
            }
            if ((threadIdx.x & 31) == 31) wsum[s][threadIdx.x >> 5] = x;
            ex[s] = x - f[s];
        }
        __syncthreads();
        unsigned tot[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            unsigned before = 0, all = 0;
            for (int w = 0; w < 8; ++w) {
                if (w < (int)(threadIdx.x >> 5)) before += wsum[s][w];
                all += wsum[s][w];
            }
            ex[s] += before + run[s] + a.boff[(size_t)s * nb + blockIdx.x];
            tot[s] = all;
        }
        __syncthreads();
        if (threadIdx.x < 3) run[threadIdx.x] += tot[threadIdx.x];
        if (i < a.n && k != 0) {
            if (f[0]) copy_gaussian(a, i, ex[0], true);
            if (f[1]) copy_gaussian(a, i, K1 + ex[1], false);
            if (f[2]) {
                const size_t d0 = K1 + K2 + 2ull * ex[2];
                copy_gaussian(a, i, d0, false);
                copy_gaussian(a, i, d0 + 1, false);
                const float* q = a.p.f[2] + 4 * (size_t)i;
                const float* ls = a.p.f[1] + 3 * (size_t)i;
                const float* mu = a.p.f[0] + 3 * (size_t)i;
                const float qn = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
                const float w = q[0] * qn, x = q[1] * qn, y = q[2] * qn, z = q[3] * qn;
                const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                                       {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                                       {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
                const float s[3] = {expf(ls[0]), expf(ls[1]), expf(ls[2])};
                for (int c = 0; c < 2; ++c) {
                    const float* nz = a.noise + 6 * (size_t)i + 3 * c;
                    const float v0 = s[0] * nz[0], v1 = s[1] * nz[1], v2 = s[2] * nz[2];
                    float* mo = a.po.f[0] + 3 * (d0 + c);
                    float* lo = a.po.f[1] + 3 * (d0 + c);
#pragma unroll
                    for (int rr = 0; rr < 3; ++rr) {
                        mo[rr] = mu[rr] + R[rr][0] * v0 + R[rr][1] * v1 + R[rr][2] * v2;
                        lo[rr] = ls[rr] - a.ln16;
                    }
                }
            }
        }
        __syncthreads();
    }
}

Fields fields_of(const le_gaussian_grads* g)
{
    Fields f;
    float* const p[7] = {g->means, g->log_scales, g->quats, g->opacity_raw, g->sh, g->feat, g->unc};
    for (int i = 0; i < 7; ++i) f.f[i] = p[i];
    return f;
}

bool fields_ok(const le_gaussian_grads* g)
{
    return g && g->means && g->log_scales && g->quats && g->opacity_raw && g->sh && g->feat && g->unc;
}

}  // namespace
}  // namespace leg

using namespace leg;

extern "C" le_status le_densify_stats(int32_t n, const float* grad2d, const int32_t* radius, float* acc, int32_t* cnt,
                                      int32_t* max_radius, void* stream)
{
    LE_TRACE("le_densify_stats");
    LE_CHECK_ARG(n >= 0, "n = %d < 0", n);
    if (n == 0) return LE_OK;
    LE_CHECK_ARG(grad2d && radius && acc && cnt, "null pointer");
    LE_CHECK_ARG(aligned16(grad2d), "grad2d must be 16-byte aligned");
    densify_stats_kernel<<<(n + 255) / 256, 256, 0, as_stream(stream)>>>(n, reinterpret_cast<const float4*>(grad2d),
                                                                         radius, acc, cnt, max_radius);
    LE_LAUNCHED();
    return LE_OK;
}

extern "C" le_status le_opacity_reset(int32_t n, float* opacity_raw, float* m_opacity, float* v_opacity,
                                      float max_opacity, void* stream)
{
    LE_TRACE("le_opacity_reset");
    LE_CHECK_ARG(n >= 0, "n = %d < 0", n);
    LE_CHECK_ARG(max_opacity > 0.f && max_opacity < 1.f, "max_opacity = %g outside (0, 1)", (double)max_opacity);
    if (n == 0) return LE_OK;
    LE_CHECK_ARG(opacity_raw && m_opacity && v_opacity, "null pointer");
    const float logit_max = (float)log((double)max_opacity / (1.0 - (double)max_opacity));
    opacity_reset_kernel<<<(n + 255) / 256, 256, 0, as_stream(stream)>>>(n, opacity_raw, m_opacity, v_opacity,
                                                                         logit_max);
    LE_LAUNCHED();
    return LE_OK;
}

extern "C" le_status le_densify_workspace(int32_t n, size_t* bytes)
{
    LE_TRACE("le_densify_workspace");
    LE_CHECK_ARG(bytes != nullptr && n >= 0, "bad arguments");
    const size_t nb = ((size_t)n + kDB - 1) / kDB;
    *bytes = ((size_t)n + 255) / 256 * 256 + (3 * nb * 4 + 255) / 256 * 256 + 256;
    return LE_OK;
}

extern "C" le_status le_densify(const le_densify_config* cfg, const le_gaussians* g, const le_gaussian_grads* m,
                                const le_gaussian_grads* v, const float* acc, const int32_t* cnt,
                                const int32_t* max_radius, const float* noise,
                                int64_t n_cap, const le_gaussian_grads* g_out, const le_gaussian_grads* m_out,
                                const le_gaussian_grads* v_out, int64_t* n_out, void* workspace,
                                size_t workspace_bytes, void* stream)
{
    LE_TRACE("le_densify");
    LE_CHECK_ARG(cfg && g && n_out, "null config / gaussians / n_out");
    LE_CHECK_ARG(g->n >= 0 && g->sh_degree >= 0 && g->sh_degree <= 3, "bad gaussians");
    LE_CHECK_ARG(cfg->min_opacity > 0.f && cfg->min_opacity < 1.f && cfg->percent_dense > 0.f &&
                     cfg->scene_extent > 0.f && cfg->grad_thresh >= 0.f && cfg->max_screen_size >= 0.f &&
                     cfg->world_frac >= 0.f,
                 "bad densify config");
    const int n = g->n;
    if (n == 0) {
        *n_out = 0;
        return LE_OK;
    }
    LE_CHECK_ARG(g->means && g->log_scales && g->quats && g->opacity_raw && g->sh && g->feat && g->unc,
                 "null Gaussian parameter");
    LE_CHECK_ARG(fields_ok(m) && fields_ok(v) && fields_ok(g_out) && fields_ok(m_out) && fields_ok(v_out),
                 "null moment / output pointer");
    LE_CHECK_ARG(acc && cnt && noise && workspace, "null statistics / noise / workspace");
    LE_CHECK_ARG(cfg->max_screen_size == 0.f || max_radius, "max_screen_size > 0 needs max_radius");
    size_t need = 0;
    le_densify_workspace(n, &need);
    LE_CHECK_ARG(workspace_bytes >= need, "workspace has %zu bytes, needs %zu", workspace_bytes, need);
    const int nb = (n + kDB - 1) / kDB;
    unsigned char* w = static_cast<unsigned char*>(workspace);
    uint8_t* kind = w;
    unsigned* bcount = reinterpret_cast<unsigned*>(w + ((size_t)n + 255) / 256 * 256);
    unsigned long long* totals =
        reinterpret_cast<unsigned long long*>(w + ((size_t)n + 255) / 256 * 256 + (3 * (size_t)nb * 4 + 255) / 256 * 256);
    DensifyThresholds t;
    t.grad_thresh = cfg->grad_thresh;
    t.log_big = (float)log((double)cfg->percent_dense * (double)cfg->scene_extent);
    t.logit_min = (float)log((double)cfg->min_opacity / (1.0 - (double)cfg->min_opacity));
    t.ln16 = (float)log(1.6);
    t.max_screen = cfg->max_screen_size;
    t.log_world = cfg->world_frac > 0.f ? (float)log((double)cfg->world_frac * (double)cfg->scene_extent) : INFINITY;
    cudaStream_t s = as_stream(stream);
    densify_count_kernel<<<nb, 256, 0, s>>>(n, g->log_scales, g->opacity_raw, acc, cnt, max_radius, t, kind,
                                            bcount);
    LE_LAUNCHED();
    densify_scan_kernel<<<1, 1024, 0, s>>>(bcount, nb, totals);
    LE_LAUNCHED();
    unsigned long long h[3];
    LE_CUDA(cudaMemcpyAsync(h, totals, sizeof(h), cudaMemcpyDeviceToHost, s));
    LE_CUDA(cudaStreamSynchronize(s));
    const unsigned long long total = h[0] + h[1] + 2 * h[2];
    *n_out = (int64_t)total;
    if ((long long)total > n_cap) {
        set_error("densify: %llu Gaussians after densification exceed the capacity %lld", total, (long long)n_cap);
        return LE_ERR_CAPACITY;
    }
    ScatterArgs a;
    a.n = n;
    a.nc = (g->sh_degree + 1) * (g->sh_degree + 1);
    float* const gp[7] = {const_cast<float*>(g->means), const_cast<float*>(g->log_scales), const_cast<float*>(g->quats),
                          const_cast<float*>(g->opacity_raw), const_cast<float*>(g->sh), const_cast<float*>(g->feat),
                          const_cast<float*>(g->unc)};
    for (int i = 0; i < 7; ++i) a.p.f[i] = gp[i];
    a.m = fields_of(m);
    a.v = fields_of(v);
    a.po = fields_of(g_out);
    a.mo = fields_of(m_out);
    a.vo = fields_of(v_out);
    a.kind = kind;
    a.boff = bcount;
    a.totals = totals;
    a.noise = noise;
    a.ln16 = t.ln16;
    densify_scatter_kernel<<<nb, 256, 0, s>>>(a);
    LE_LAUNCHED();
    return LE_OK;
}
