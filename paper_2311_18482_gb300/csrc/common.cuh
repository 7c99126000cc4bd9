// Internal helpers shared by the CUDA translation units of libleg.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <nvtx3/nvToolsExt.h>

#include "../../include/leg.h"

namespace leg {

// Named NVTX range around a C-ABI call (shows up on profiler timelines; a
// no-op unless a tool is attached).
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};
#define LE_TRACE(name) ::leg::TraceRange le_trace_range_(name)


// Per-thread error message and launch counter (host side).
void set_error(const char* fmt, ...);
void count_launch(int n = 1);

#define LE_CHECK_ARG(cond, ...)                 \
    do {                                        \
        if (!(cond)) {                          \
            ::leg::set_error(__VA_ARGS__);      \
            return LE_ERR_INVALID_ARG;          \
        }                                       \
    } while (0)

#define LE_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) {                                                        \
            ::leg::set_error("%s failed: %s", #call, cudaGetErrorString(e_));           \
            return LE_ERR_CUDA;                                                         \
        }                                                                               \
    } while (0)

// After a kernel launch: record it and check for launch errors.
#define LE_LAUNCHED()                                                                   \
    do {                                                                                \
        ::leg::count_launch();                                                          \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess) {                                                        \
            ::leg::set_error("kernel launch failed at %s:%d: %s", __FILE__, __LINE__,    \
                             cudaGetErrorString(e_));                                   \
            return LE_ERR_CUDA;                                                         \
        }                                                                               \
    } while (0)

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }
inline int tiles_x(const le_camera* c) { return (c->width + LE_TILE - 1) / LE_TILE; }
inline int tiles_y(const le_camera* c) { return (c->height + LE_TILE - 1) / LE_TILE; }
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Tile rows per placement block (binning) -- also the granularity of the lazy
// placement's row-group flags written by the compositing phases.
#define LE_PLACE_ROWS 2

// 2^x on the special-function unit (approximate, flush-to-zero).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The splat record stores the conic in base-2 exponent units, so that
// alpha = o 2^-q with q = A' dx^2 + B' dx dy + C' dy^2 (kConicScale*: A' = A log2(e)/2,
// B' = B log2(e), C' = C log2(e)/2).  kConicUnscale* undo it.
constexpr float kConicScaleAC = 0.72134752044448170f, kConicScaleB = 1.4426950408889634f;
constexpr float kConicUnscaleAC = 1.3862943611198906f, kConicUnscaleB = 0.69314718055994531f;

// Adam (Kingma & Ba; Sec. 4 trains with it) with both bias corrections folded
// in: step_size = lr / (1 - b1^t), inv_sqrt_c2 = 1 / sqrt(1 - b2^t); c1 = 1 - b1,
// c2 = 1 - b2 (FP32).
struct AdamParams {
    float b1, b2, c1, c2, step_size, inv_sqrt_c2, eps;
};

// sqrt(x) and 1/x on the special-function unit (approximate: a relative error
// of a few 2^-23, far inside the step's own FP32 noise; x >= 0, resp. x >= eps).
__device__ __forceinline__ float sqrt_approx(float x)
{
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One element: m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
// p <- clamp(p - step_size m / (sqrt(v) inv_sqrt_c2 + eps), lo, hi).  A fixed
// sequence of operations (the moments in IEEE FP32, the denominator's square
// root and reciprocal on the SFU), so every kernel that applies it -- scalar
// or four elements at a time (adam_step4) -- agrees bit for bit.
__device__ __forceinline__ float adam_step(float p, float g, float& m, float& v, const AdamParams& h, float lo,
                                           float hi)
{
    m = __fmaf_rn(h.b1, m, __fmul_rn(h.c1, g));
    v = __fmaf_rn(h.b2, v, __fmul_rn(__fmul_rn(h.c2, g), g));
    const float den = __fmaf_rn(sqrt_approx(v), h.inv_sqrt_c2, h.eps);
    return fminf(fmaxf(__fmaf_rn(-__fmul_rn(h.step_size, m), rcp_approx(den), p), lo), hi);
}

// adam_step on (x, y) with paired FP32 instructions: per component the same
// IEEE operations as the scalar form.
__device__ __forceinline__ float2 adam_step2(float2 p, float2 g, float2& m, float2& v, const AdamParams& h, float lo,
                                             float hi)
{
    m = __ffma2_rn(make_float2(h.b1, h.b1), m, __fmul2_rn(make_float2(h.c1, h.c1), g));
    v = __ffma2_rn(make_float2(h.b2, h.b2), v, __fmul2_rn(__fmul2_rn(make_float2(h.c2, h.c2), g), g));
    const float2 den = __ffma2_rn(make_float2(sqrt_approx(v.x), sqrt_approx(v.y)),
                                  make_float2(h.inv_sqrt_c2, h.inv_sqrt_c2), make_float2(h.eps, h.eps));
    const float2 sm = __fmul2_rn(make_float2(h.step_size, h.step_size), m);
    const float2 r = __ffma2_rn(make_float2(-sm.x, -sm.y), make_float2(rcp_approx(den.x), rcp_approx(den.y)), p);
    return make_float2(fminf(fmaxf(r.x, lo), hi), fminf(fmaxf(r.y, lo), hi));
}

// Four consecutive elements (two pairs).
__device__ __forceinline__ void adam_step4(float4& p, float4 g, float4& m, float4& v, const AdamParams& h, float lo,
                                           float hi)
{
    float2 ma = make_float2(m.x, m.y), mb = make_float2(m.z, m.w);
    float2 va = make_float2(v.x, v.y), vb = make_float2(v.z, v.w);
    const float2 pa = adam_step2(make_float2(p.x, p.y), make_float2(g.x, g.y), ma, va, h, lo, hi);
    const float2 pb = adam_step2(make_float2(p.z, p.w), make_float2(g.z, g.w), mb, vb, h, lo, hi);
    p = make_float4(pa.x, pa.y, pb.x, pb.y);
    m = make_float4(ma.x, ma.y, mb.x, mb.y);
    v = make_float4(va.x, va.y, vb.x, vb.y);
}

AdamParams adam_params(int32_t step, float lr, float beta1, float beta2, float eps);

// Camera values the kernels need, passed by value.
struct CamParams {
    float view[12];
    float campos[3];
    float fx, fy, cx, cy;
    int W, H, TX, TY;
    float near_z;
    float bg[3];
};

inline CamParams cam_params(const le_camera* c)
{
    CamParams p;
    for (int i = 0; i < 12; ++i) p.view[i] = c->view[i];
    for (int i = 0; i < 3; ++i) p.campos[i] = c->campos[i];
    p.fx = c->fx;
    p.fy = c->fy;
    p.cx = c->cx;
    p.cy = c->cy;
    p.W = c->width;
    p.H = c->height;
    p.TX = tiles_x(c);
    p.TY = tiles_y(c);
    p.near_z = c->near_z;
    for (int i = 0; i < 3; ++i) p.bg[i] = c->bg[i];
    return p;
}

inline le_status check_camera(const le_camera* c)
{
    LE_CHECK_ARG(c != nullptr, "camera is null");
    LE_CHECK_ARG(c->width > 0 && c->height > 0 && c->width <= 16384 && c->height <= 16384,
                 "camera size %dx%d out of range", c->width, c->height);
    LE_CHECK_ARG(c->fx > 0.f && c->fy > 0.f, "focal lengths must be positive");
    return LE_OK;
}

}  // namespace leg
