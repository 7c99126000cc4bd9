// tcgen05 / TMEM / mbarrier building blocks (inline PTX, sm_100-family).
//
// Shared-memory operands use the no-swizzle canonical layout: a bf16 matrix
// X[r][c] with C columns is stored as 8x8 core matrices of 8 rows x 16 bytes,
//   off(r, c) = (r/8) * (C/8) * 128 + (c/8) * 128 + (r%8) * 16 + (c%8) * 2.
// Read K-major (rows = M or N, columns = K) its descriptor has LBO = 128 (core
// stride along K) and SBO = (C/8)*128 (stride between 8-row groups); read
// MN-major (rows = K, columns = M or N) LBO = (C/8)*128 (stride along K) and
// SBO = 128.  In both cases LBO is the stride between core matrices adjacent
// in K and SBO the one between core matrices adjacent in M/N.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace leg {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Named barrier over `n` threads; returns whether any participating thread passed pred = true.
__device__ __forceinline__ bool bar_any(int id, int n, bool pred)
{
    uint32_t r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}\n"
                 : "=r"(r)
                 : "r"((uint32_t)pred), "r"(id), "r"(n)
                 : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}

// Bounded wait for the phase with the given parity to complete.  Gives up
// after ~2^31 SM cycles (about a second) and returns false.  The try_wait
// carries a suspend-time hint, so the waiting thread sleeps in the barrier
// until the phase completes instead of spinning on issue slots.
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity)
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

__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> this CTA's shared memory, completion counted on m.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* m)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(m))
                 : "memory");
}

// 2-D tensor store shared -> global through the tensor map (TMA), counted in
// this thread's bulk async-group; elements outside the tensor are not written.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, const void* src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}

// 1-D bulk copy this CTA's shared memory -> global, counted in this thread's
// bulk async-group (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Until this thread's committed bulk stores have read their shared-memory source.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Until this thread's committed bulk stores have completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Warp-wide TMEM allocation; the base address is written to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// kind::f16 instruction descriptor: BF16 A and B, FP32 accumulator, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int N, bool a_mn, bool b_mn)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ uint64_t make_desc(uint32_t start, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((start & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// D[tmem] (+)= A * B, issued by one thread.
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                     d_tmem),
                 "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
                 : "memory");
}

// mbarrier arrives once all tcgen05 operations issued so far by this thread complete.
__device__ __forceinline__ void commit(uint64_t* m)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(m))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.  The load and its
// wait are one asm statement, so no use of the registers can be scheduled
// before the data has arrived.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "{\ntcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n}\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Store 16 FP32 values to consecutive columns of this thread's TMEM lane; call
// tmem_wait_st() before reading them back.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v)
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
        "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
        "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Store one FP32 value to a column of this thread's TMEM lane.
__device__ __forceinline__ void tmem_st1(uint32_t taddr, float v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(taddr), "r"(__float_as_uint(v)) : "memory");
}

// Single arrival on an mbarrier (release semantics at CTA scope).
__device__ __forceinline__ void mbar_arrive(uint64_t* m)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(m)) : "memory");
}


// ---------------------------------------------------------------------------
// Canonical no-swizzle bf16 buffer in shared memory.
struct SBuf {
    unsigned char* p;
    int C;   // columns (multiple of 8)
};

__host__ __device__ constexpr uint32_t sbuf_bytes(int R, int C) { return (uint32_t)R * C * 2; }

__device__ __forceinline__ uint32_t sbuf_off(int r, int c, int C)
{
    return (uint32_t)((r >> 3) * (C >> 3) * 128 + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// 8 consecutive columns [c0, c0+8) of row r (c0 multiple of 8) in one 16-byte store.
__device__ __forceinline__ void sbuf_store8(const SBuf& b, int r, int c0, const float* v)
{
    __nv_bfloat162 h[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    *reinterpret_cast<uint4*>(b.p + sbuf_off(r, c0, b.C)) = *reinterpret_cast<uint4*>(h);
}

__device__ __forceinline__ void sbuf_load8(const SBuf& b, int r, int c0, float* v)
{
    const uint4 u = *reinterpret_cast<const uint4*>(b.p + sbuf_off(r, c0, b.C));
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(h[j]);
        v[2 * j] = f.x;
        v[2 * j + 1] = f.y;
    }
}

// Descriptor of the (128-row or N-row) K-major block whose first row is row0,
// K columns starting at k0 (both multiples of 8).
__device__ __forceinline__ uint64_t kdesc(const SBuf& b, int row0, int k0)
{
    return make_desc(smem_u32(b.p) + sbuf_off(row0, k0, b.C), 128u, (uint32_t)(b.C >> 3) * 128u);
}

// Descriptor of the MN-major block: rows are K (starting at k0), columns are M/N
// (starting at mn0).
__device__ __forceinline__ uint64_t mndesc(const SBuf& b, int k0, int mn0)
{
    return make_desc(smem_u32(b.p) + sbuf_off(k0, mn0, b.C), (uint32_t)(b.C >> 3) * 128u, 128u);
}

// The same for a buffer given by its shared-memory address and column count.
__device__ __forceinline__ uint64_t kdesc_at(uint32_t base, int C, int row0, int k0)
{
    return make_desc(base + sbuf_off(row0, k0, C), 128u, (uint32_t)(C >> 3) * 128u);
}

__device__ __forceinline__ uint64_t mndesc_at(uint32_t base, int C, int k0, int mn0)
{
    return make_desc(base + sbuf_off(k0, mn0, C), (uint32_t)(C >> 3) * 128u, 128u);
}

// 8 floats -> 8 bf16 in one 16-byte shared store at a shared-memory address.
__device__ __forceinline__ void sts_bf16x8(uint32_t addr, const float* v)
{
    __nv_bfloat162 h[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
    const uint4 u = *reinterpret_cast<uint4*>(h);
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(u.x), "r"(u.y), "r"(u.z), "r"(u.w)
                 : "memory");
}

// Hide a value's origin from the optimiser, so that what is derived from it is
// recomputed where used instead of being kept live across a loop.
__device__ __forceinline__ uint32_t opaque(uint32_t x)
{
    asm volatile("" : "+r"(x));
    return x;
}

// Fill rows [0,R) x cols [0,C) of a canonical buffer from fp32 row-major src
// (src[r*ld + c], zero outside [0,rs) x [0,cs)); all threads of the block.
__device__ __forceinline__ void sbuf_fill(const SBuf& b, int R, const float* src, int ld, int rs, int cs)
{
    const int chunks = R * (b.C >> 3);
    for (int i = threadIdx.x; i < chunks; i += blockDim.x) {
        const int r = i / (b.C >> 3), c0 = (i % (b.C >> 3)) * 8;
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (r < rs && c0 + j < cs) ? src[(size_t)r * ld + c0 + j] : 0.f;
        sbuf_store8(b, r, c0, v);
    }
}

// cuTensorMapEncodeTiled from the driver (once per process).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline le_status tensor_map_encoder(EncodeTiled* fn)
{
    static EncodeTiled cached = nullptr;
    if (!cached) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) !=
                cudaSuccess ||
            qr != cudaDriverEntryPointSuccess || !p) {
            set_error("cuTensorMapEncodeTiled is not available from the driver");
            return LE_ERR_CUDA;
        }
        cached = reinterpret_cast<EncodeTiled>(p);
    }
    *fn = cached;
    return LE_OK;
}

}  // namespace tc
}  // namespace leg
