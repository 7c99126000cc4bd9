// Tile binning: 64-bit (tile | depth) keys, their stable order and the per-tile
// ranges of the 3DGS rasterizer the paper reuses (Sec. 4).
//
// A Gaussian is copied to the tiles of its rectangle that its tile ellipse
// reaches (row_span below; the ellipse comes from the key path of
// le_preprocess and is not in the paper): the renderer would skip it on every
// pixel of the other tiles, so they only cost time.
//
// The order is that of a stable sort of key = (tile_id << 32) | bits(depth)
// over the copies emitted Gaussian by Gaussian: inside each tile, copies are
// ordered by depth, ties by Gaussian index.  It is computed without sorting the
// K copies at all:
//   1. e[i] = bits(depth_i) << 32 | i          (culled: 0xFFFFFFFF, sorted last)
//   2. stable LSD radix sort of e on bits 32..63 (4 passes over the N Gaussians,
//      each count / scan / scatter, see depth_sort)
//   3. split the depth-sorted Gaussians into chunks; per chunk, the number of
//      copies in every tile from per-row difference arrays of the row spans
//   4. one exclusive scan of those counts in tile-major order: entry (t, c) is
//      where chunk c's copies of tile t start; the total is K; consecutive
//      tiles' first entries are the tile ranges
//   5. blocks of (8 tile rows x a super-chunk of Gaussians) write the copies in
//      depth order through per-tile cursors held in registers (one warp per
//      row, one lane per 32nd tile of the row).
// No kernel waits on another block.
#include "common.cuh"

namespace leg {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;   // 4096 elements per block
constexpr int kWarps = kThreads / 32;

// ----------------------------------------------------------------------------
// Exclusive scan of u32 (2 kernels: per-block sums, then each block adds the
// sums of the blocks before it to its own exclusive prefix).  `In` yields element i.

struct DirectIn {
    const uint32_t* p;
    __device__ uint32_t operator()(int i) const { return p[i]; }
};

template <int NW = kWarps>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums, uint32_t* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < NW ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NW) warp_sums[lane] = s;
    }
    __syncthreads();
    const uint32_t before = (w > 0 ? warp_sums[w - 1] : 0u) + x - v;
    if (total) *total = warp_sums[NW - 1];
    return before;
}

template <class In>
__global__ void __launch_bounds__(kThreads) scan_reduce_kernel(In in, int n, uint32_t* partials)
{
    __shared__ uint32_t ws[kWarps];
    const int base = blockIdx.x * kTile;
    uint32_t s = 0;
    for (int k = 0; k < kItems; ++k) {
        const int i = base + k * kThreads + threadIdx.x;
        if (i < n) s += in(i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kWarps; ++w) t += ws[w];
        partials[blockIdx.x] = t;
    }
}

// out[i] = (sum of the partials of the blocks before this one) + exclusive
// prefix of in within the block; the last block also writes the total.  out
// may alias in.
template <class In>
__global__ void __launch_bounds__(kThreads) scan_apply_kernel(In in, int n, uint32_t* out, const uint32_t* partials,
                                                             uint32_t* total)
{
    __shared__ uint32_t sm[kTile + kTile / 32];
    __shared__ uint32_t ws[kWarps];
    __shared__ uint32_t s_off;
    const int base = blockIdx.x * kTile;
    {
        uint32_t p = 0;
        for (int b = threadIdx.x; b < (int)blockIdx.x; b += kThreads) p += partials[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = p;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < kWarps; ++w) t += ws[w];
            s_off = t;
            if (blockIdx.x == gridDim.x - 1) *total = t + partials[blockIdx.x];
        }
        __syncthreads();
    }
    for (int k = 0; k < kItems; ++k) {
        const int j = k * kThreads + threadIdx.x;
        const int i = base + j;
        sm[j + (j >> 5)] = i < n ? in(i) : 0u;
    }
    __syncthreads();
    uint32_t v[kItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int j = threadIdx.x * kItems + k;
        v[k] = sm[j + (j >> 5)];
        s += v[k];
    }
    uint32_t run = block_exclusive_scan(s, ws, nullptr) + s_off;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const int j = threadIdx.x * kItems + k;
        sm[j + (j >> 5)] = run;
        run += v[k];
    }
    __syncthreads();
    for (int k = 0; k < kItems; ++k) {
        const int j = k * kThreads + threadIdx.x;
        const int i = base + j;
        if (i < n) out[i] = sm[j + (j >> 5)];
    }
}

template <class In>
le_status exclusive_scan(In in, int n, uint32_t* out, uint32_t* partials, uint32_t* total, cudaStream_t s)
{
    const int nb = (n + kTile - 1) / kTile;
    if (nb > 1024 * 16) {
        set_error("scan of %d elements exceeds the supported size", n);
        return LE_ERR_CAPACITY;
    }
    scan_reduce_kernel<In><<<nb, kThreads, 0, s>>>(in, n, partials);
    LE_LAUNCHED();
    scan_apply_kernel<In><<<nb, kThreads, 0, s>>>(in, n, out, partials, total);
    LE_LAUNCHED();
    return LE_OK;
}

// ----------------------------------------------------------------------------
// Depth sort: stable LSD radix sort of e = bits(depth) << 32 | index on bits
// 32-63 in four 8-bit passes.  Each pass is count / scan / scatter over tiles
// of kSortTile consecutive elements, and no block waits on another:
//   count    per-tile digit counts, counts[d][b] (digit-major, rows padded to
//            a multiple of 4), and the digits' totals (pass 0's are counted
//            while the keys are built);
//   rowscan  one warp per digit: the exclusive prefix of its row plus the
//            digit's base (the totals of all smaller digits), so counts[d][b]
//            becomes the first output position of tile b's digit-d elements;
//   scatter  each tile ranks its elements stably (warp-private digit counters,
//            warps in element order) and writes them to their positions.
// The last scatter also gathers each Gaussian's rectangle and tile ellipse
// into depth order (zero for culled Gaussians) for the kernels that follow.
constexpr int kSortPasses = 4;
constexpr int kSortThreads = 512;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096 elements per tile
constexpr int kSortWarps = kSortThreads / 32;

__device__ __forceinline__ uint32_t digit_of(uint64_t e, int shift) { return (uint32_t)(e >> shift) & 255u; }

__host__ __device__ constexpr int sort_tiles(int n) { return (n + kSortTile - 1) / kSortTile; }
__host__ __device__ constexpr int sort_row(int n) { return (sort_tiles(n) + 3) / 4 * 4; }

// Tile b's digit counts from shared memory to counts[d][b] and the totals.
__device__ __forceinline__ void publish_counts(const uint32_t* h, uint32_t* counts, int row, uint32_t* totals)
{
    if (threadIdx.x < 256) {
        const uint32_t c = h[threadIdx.x];
        counts[(size_t)threadIdx.x * row + blockIdx.x] = c;
        if (c) atomicAdd(totals + threadIdx.x, c);
    }
}

// e[i] (culled: 0xFFFFFFFF in the high word, sorted last) and pass 0's counts.
__global__ void __launch_bounds__(kSortThreads) depth_elems_kernel(int n, const float* __restrict__ depth,
                                                                   const int* __restrict__ tiles,
                                                                   uint64_t* __restrict__ e, uint32_t* counts,
                                                                   int row, uint32_t* totals)
{
    __shared__ uint32_t h[256];
    if (threadIdx.x < 256) h[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const int i = blockIdx.x * kSortTile + k * kSortThreads + threadIdx.x;
        if (i < n) {
            const uint32_t hi = tiles[i] > 0 ? __float_as_uint(depth[i]) : 0xFFFFFFFFu;
            e[i] = ((uint64_t)hi << 32) | (uint32_t)i;
            atomicAdd(&h[hi & 255u], 1u);
        }
    }
    __syncthreads();
    publish_counts(h, counts, row, totals);
}

// Per-tile counts of the digit (e >> shift) & 255.
__global__ void __launch_bounds__(kSortThreads) sort_count_kernel(const uint64_t* __restrict__ in, int n, int shift,
                                                                  uint32_t* counts, int row, uint32_t* totals)
{
    __shared__ uint32_t h[256];
    if (threadIdx.x < 256) h[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const int i = blockIdx.x * kSortTile + k * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[digit_of(in[i], shift)], 1u);
    }
    __syncthreads();
    publish_counts(h, counts, row, totals);
}

// counts[d][0..nt) -> base(d) + exclusive prefix along the row, one warp per
// digit d; base(d) = the totals of digits 0..d-1.  Lanes own 8 consecutive
// entries (two 16-byte accesses) per round of 256.
__global__ void __launch_bounds__(256) sort_rowscan_kernel(uint32_t* counts, int nt, int row,
                                                           const uint32_t* __restrict__ totals)
{
    const int lane = threadIdx.x & 31;
    const int d = blockIdx.x * 8 + (threadIdx.x >> 5);
    uint32_t base = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int dd = lane * 8 + k;
        base += dd < d ? totals[dd] : 0u;
    }
    base = __reduce_add_sync(0xffffffffu, base);
    uint32_t* r = counts + (size_t)d * row;
    for (int b0 = 0; b0 < nt; b0 += 256) {
        const int b = b0 + lane * 8;
        uint4 v0 = make_uint4(0, 0, 0, 0), v1 = make_uint4(0, 0, 0, 0);
        if (b < row) v0 = *reinterpret_cast<const uint4*>(r + b);
        if (b + 4 < row) v1 = *reinterpret_cast<const uint4*>(r + b + 4);
        uint32_t x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t c = b + k < nt ? x[k] : 0u;
            x[k] = sum;
            sum += c;
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t off = base + incl - sum;
        if (b < row) *reinterpret_cast<uint4*>(r + b) = make_uint4(off + x[0], off + x[1], off + x[2], off + x[3]);
        if (b + 4 < row)
            *reinterpret_cast<uint4*>(r + b + 4) = make_uint4(off + x[4], off + x[5], off + x[6], off + x[7]);
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// Rectangles and tile ellipses of the depth-sorted Gaussians (the last pass).
struct SortGather {
    const int* tiles;
    const ushort4* rect;
    const float4* ell;
    ushort4* drect;
    float4* dell;
};

// One pass on digit (e >> shift) & 255 from in to out; offsets: counts after
// sort_rowscan_kernel.  gather.drect non-null: also gather into depth order.
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(const uint64_t* __restrict__ in,
                                                                    uint64_t* __restrict__ out, int n, int shift,
                                                                    const uint32_t* __restrict__ offsets, int row,
                                                                    SortGather gather)
{
    __shared__ uint64_t stage[kSortTile];
    __shared__ uint32_t warp_cnt[kSortWarps][256];
    __shared__ uint32_t gbase[256], lbase[256];
    __shared__ uint32_t ws[kSortWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < kSortWarps * 256; j += kSortThreads) (&warp_cnt[0][0])[j] = 0;
    if (threadIdx.x < 256) gbase[threadIdx.x] = offsets[(size_t)threadIdx.x * row + blockIdx.x];
    __syncthreads();
    const int base = blockIdx.x * kSortTile;
    const int cnt = min(kSortTile, n - base);

    // each warp owns the contiguous sub-range [w * 256, (w + 1) * 256) of the tile
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t e[kSortItems];
    uint32_t dg[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const int j = w * (kSortTile / kSortWarps) + k * 32 + lane;
        const bool valid = j < cnt;
        e[k] = valid ? in[base + j] : 0ull;
        dg[k] = valid ? digit_of(e[k], shift) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const uint32_t vm = __ballot_sync(0xffffffffu, dg[k] != 0xFFFFFFFFu);
        if (dg[k] != 0xFFFFFFFFu) {
            const uint32_t peers = __match_any_sync(vm, dg[k]);
            if (lane == __ffs(peers) - 1) warp_cnt[w][dg[k]] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit (thread d): exclusive prefix over warps, the tile's count, and the
    // tile-local start of the digit's run
    uint32_t tot = 0;
    if (threadIdx.x < 256) {
        const int d = threadIdx.x;
        for (int ww = 0; ww < kSortWarps; ++ww) {
            const uint32_t v = warp_cnt[ww][d];
            warp_cnt[ww][d] = tot;
            tot += v;
        }
    }
    const uint32_t lb = block_exclusive_scan<kSortWarps>(tot, ws, nullptr);
    if (threadIdx.x < 256) lbase[threadIdx.x] = lb;
    __syncthreads();
    // stage the tile's elements in digit order (stable), then write them out
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const bool valid = dg[k] != 0xFFFFFFFFu;
        const uint32_t vm = __ballot_sync(0xffffffffu, valid);
        uint32_t peers = 0, pos = 0;
        if (valid) {
            peers = __match_any_sync(vm, dg[k]);
            pos = lbase[dg[k]] + warp_cnt[w][dg[k]] + __popc(peers & lt);
        }
        __syncwarp();
        if (valid) {
            if (lane == __ffs(peers) - 1) warp_cnt[w][dg[k]] += __popc(peers);
            stage[pos] = e[k];
        }
        __syncwarp();
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cnt; j += kSortThreads) {
        const uint64_t v = stage[j];
        const uint32_t d = digit_of(v, shift);
        const uint32_t p = gbase[d] + (j - lbase[d]);
        out[p] = v;
        if (gather.drect) {
            const uint32_t gid = (uint32_t)v;
            uint2 r = make_uint2(0u, 0u);
            float4 e0 = make_float4(0.f, 0.f, 0.f, 0.f), e1 = e0;
            if (gather.tiles[gid] > 0) {
                r = reinterpret_cast<const uint2*>(gather.rect)[gid];
                e0 = gather.ell[2 * (size_t)gid];
                e1 = gather.ell[2 * (size_t)gid + 1];
            }
            reinterpret_cast<uint2*>(gather.drect)[p] = r;
            gather.dell[2 * (size_t)p] = e0;
            gather.dell[2 * (size_t)p + 1] = e1;
        }
    }
}

// Tiles [xl, xr) of rectangle row ty that the tile ellipse {e0, e1} reaches.
// The ellipse is convex, so its tiles in a row are contiguous.  For the row's
// band of pixel-centre offsets dy in [lo, hi], the right end s dy + sqrt(k (mm -
// dy^2)) of a row is concave in dy with its peak at ystar, so the band's
// right-most point is at clamp(ystar, lo, hi), its left-most (mirror image) at
// clamp(-ystar, lo, hi).  Every operation is an explicit IEEE FP32 one, in a
// fixed order, so that every implementation gets the same integers.
__device__ __forceinline__ void row_span(const float4 e0, const float4 e1, const ushort4 r, int ty, int& xl, int& xr)
{
    xl = xr = r.x;
    const float yc = __fsub_rn((float)(16 * ty), e0.y);
    const float lo = __fsub_rn(yc, e1.w);
    const float hi = __fadd_rn(__fadd_rn(yc, 15.0f), e1.w);
    const float dR = fminf(fmaxf(e1.y, lo), hi);
    const float dL = fminf(fmaxf(-e1.y, lo), hi);
    const float vR = __fsub_rn(e1.x, __fmul_rn(dR, dR));
    const float vL = __fsub_rn(e1.x, __fmul_rn(dL, dL));
    if (!(vR >= 0.0f) || !(vL >= 0.0f)) return;
    const float R = __fadd_rn(__fmul_rn(e0.z, dR), __fsqrt_rn(__fmul_rn(e0.w, vR)));
    const float L = __fsub_rn(__fmul_rn(e0.z, dL), __fsqrt_rn(__fmul_rn(e0.w, vL)));
    const float fl = ceilf(__fmul_rn(__fsub_rn(__fsub_rn(__fadd_rn(e0.x, L), e1.z), 15.0f), 0.0625f));
    const float fr = __fadd_rn(floorf(__fmul_rn(__fadd_rn(__fadd_rn(e0.x, R), e1.z), 0.0625f)), 1.0f);
    const float x0 = (float)r.x, x1 = (float)r.z;
    xl = (int)fminf(fmaxf(fl, x0), x1);
    xr = (int)fminf(fmaxf(fr, x0), x1);
    if (xr < xl) xr = xl;
}

// Copies of chunk c (depth-sorted Gaussians [c*chunk, (c+1)*chunk)) per tile
// (512 threads per block, about two Gaussians each: 256 threads, four each,
// took bin + render 0.556 against 0.536 ms at 1M Gaussians),
// via per-row difference arrays in shared memory: +1 / -1 at both ends of every
// row span, then a prefix sum along each row.  Written tile-major:
// counts[t * nchunks + c].
__global__ void __launch_bounds__(512) chunk_count_kernel(int n, const ushort4* __restrict__ drect,
                                                          const float4* __restrict__ dell, int TX, int TY,
                                                          int chunk, int nchunks, uint32_t* __restrict__ counts)
{
    extern __shared__ __align__(16) int diff[];
    const int W1 = TX + 1, cells = W1 * TY;
    // zeroed with 16-byte stores (the launch rounds the array up to whole int4s)
    for (int i = threadIdx.x; i < (cells + 3) / 4; i += blockDim.x)
        reinterpret_cast<int4*>(diff)[i] = make_int4(0, 0, 0, 0);
    __syncthreads();
    const int j0 = blockIdx.x * chunk, j1 = min(n, j0 + chunk);
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        const ushort4 r = drect[j];
        if (r.z <= r.x) continue;
        const float4 e0 = dell[2 * j], e1 = dell[2 * j + 1];
        for (int ty = r.y; ty < r.w; ++ty) {
            int xl, xr;
            row_span(e0, e1, r, ty, xl, xr);
            if (xr > xl) {
                atomicAdd(&diff[ty * W1 + xl], 1);
                atomicAdd(&diff[ty * W1 + xr], -1);
            }
        }
    }
    __syncthreads();
    // inclusive prefix sum along each row (one warp per row, 32 cells a step),
    // each cell's count written straight to its (tile, chunk) entry
    const int lane = threadIdx.x & 31;
    for (int y = threadIdx.x >> 5; y < TY; y += blockDim.x >> 5) {
        int carry = 0;
        for (int x0 = 0; x0 < TX; x0 += 32) {
            const int x = x0 + lane;
            int v = x < TX ? diff[y * W1 + x] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += t;
            }
            v += carry;
            if (x < TX) counts[(size_t)(y * TX + x) * nchunks + blockIdx.x] = (uint32_t)v;
            carry = __shfl_sync(0xffffffffu, v, 31);
        }
    }
}

// Placement.  Block (g, C): tile rows [R g, R g + R) (R = kPlaceRows) and the
// Gaussians of super-chunk C (count chunks [C*cs, (C+1)*cs)).  Each warp owns one
// row and one segment of 32 tile columns (NS segments per row); the cursor of
// tile (row, tx) starts at base[t * nchunks + C*cs] -- the exclusive scan of the
// counts in tile-major order -- and lives in a register of lane tx % 32 of the
// row's warp for that segment, so no two threads share a cursor and no barrier
// is needed between Gaussians.  Per round the block compacts, in depth order,
// the super-chunk's Gaussians whose rectangle meets its rows, computes each
// (row, Gaussian) tile span once into shared memory, and every warp then walks
// the spans of its row that meet its segment, in depth order, each lane writing
// the copies of its tile.  Only one cursor per (tile, block) advances at a time,
// so the partly written output sectors stay few enough to remain in L2.  Two
// rows per block give the first lazy phase (the nearest few chunks, every tile
// row) enough blocks to fill the GPU.  Only the tiles that receive copies in
// the block's super-chunk (an active tile with a non-empty count) do work: the
// compaction keeps the Gaussians whose rectangle reaches the column range of
// such tiles in one of the block's rows, spans are computed for those rows
// only, and a warp without such a tile skips the walk (bin + render at 1M
// Gaussians 0.602 -> 0.577 ms; the placed lists are unchanged).
constexpr int kPlaceRows = LE_PLACE_ROWS;   // tile rows per block

template <int NS>
struct PlaceShape {
    static constexpr int kThreads = 32 * kPlaceRows * NS;
    // Gaussians per thread per compaction round: the largest power of two <= 8
    // that keeps a round within 1024 Gaussians
    static constexpr int kItems = 1024 / kThreads >= 8 ? 8 : (1024 / kThreads >= 4 ? 4 : (1024 / kThreads >= 2 ? 2 : 1));
    static constexpr int kBatch = kItems * kThreads;
};

// tile_act / rows_act (nullable): only tiles with a non-zero flag get copies,
// blocks of row groups without one return at once; super-chunk blockIdx.y is
// super_base + blockIdx.y.
template <int NS>
__global__ void __launch_bounds__(PlaceShape<NS>::kThreads) place_kernel(
    int n, const uint64_t* __restrict__ dsorted, const ushort4* __restrict__ drect, const float4* __restrict__ dell,
    const float* __restrict__ depth, int TX, int TY, int super_chunk, int cstride, int nchunks,
    const uint32_t* __restrict__ base, uint32_t* __restrict__ ids, uint64_t* __restrict__ keys,
    const uint8_t* __restrict__ tile_act, const uint8_t* __restrict__ rows_act, int super_base,
    uint8_t* __restrict__ zero_a, int zero_na, uint8_t* __restrict__ zero_r, int zero_nr)
{
    using S = PlaceShape<NS>;
    // block (0, 0) clears the flags the phase's render will set (16-byte aligned arrays)
    if (zero_a && blockIdx.x == 0 && blockIdx.y == 0) {
        for (int i = threadIdx.x; i < (zero_na + 15) / 16; i += blockDim.x)
            reinterpret_cast<uint4*>(zero_a)[i] = make_uint4(0u, 0u, 0u, 0u);
        for (int i = threadIdx.x; i < (zero_nr + 15) / 16; i += blockDim.x)
            reinterpret_cast<uint4*>(zero_r)[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (rows_act && !rows_act[blockIdx.x]) return;
    __shared__ uint32_t sg[S::kBatch], sj[S::kBatch];
    __shared__ ushort4 sr[S::kBatch];
    __shared__ uint32_t span[kPlaceRows][S::kBatch];   // xl | xr << 16 of the row's tiles, 0 = none
    __shared__ uint32_t ws[S::kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rloc = warp / NS, seg = warp % NS;
    const int rb = blockIdx.x * kPlaceRows, re = min(TY, rb + kPlaceRows);
    const int row = rb + rloc;
    const bool row_ok = row < TY;
    const int C = super_base + blockIdx.y;
    const int tx = 32 * seg + lane;
    const bool mine = row_ok && tx < TX && (!tile_act || tile_act[row * TX + tx]);
    const size_t tb = (size_t)(row * TX + tx) * nchunks;
    uint32_t ctr = mine ? base[tb + (size_t)C * cstride] : 0u;
    // a block none of whose tiles has a copy in this super-chunk has nothing to place
    // (the scan holds K at the end, so the last tile's end offset is there too)
    const uint32_t cend = mine ? base[tb + (size_t)min((C + 1) * cstride, nchunks)] : 0u;
    // the tiles that receive copies here, and per row of the block the column
    // range they span: only Gaussians reaching such a range are compacted, only
    // those rows' spans computed, only warps with such a tile walk them
    const bool work = cend > ctr;
    __shared__ int s_xlo[kPlaceRows], s_xhi[kPlaceRows];
    if (threadIdx.x < kPlaceRows) {
        s_xlo[threadIdx.x] = 1 << 30;
        s_xhi[threadIdx.x] = -1;
    }
    __syncthreads();
    const int wlo = __reduce_min_sync(0xffffffffu, work ? tx : 1 << 30);
    const int whi = __reduce_max_sync(0xffffffffu, work ? tx + 1 : -1);
    if (lane == 0 && whi > 0) {
        atomicMin(&s_xlo[rloc], wlo);
        atomicMax(&s_xhi[rloc], whi);
    }
    if (!__syncthreads_or(work)) return;
    int xlo[kPlaceRows], xhi[kPlaceRows];
#pragma unroll
    for (int k = 0; k < kPlaceRows; ++k) {
        xlo[k] = s_xlo[k];
        xhi[k] = s_xhi[k];
    }
    const int j0 = C * super_chunk, j1 = min(n, j0 + super_chunk);
    for (int jb = j0; jb < j1; jb += S::kBatch) {
        // compaction: the round's Gaussians whose rectangle meets this block's
        // rows, in depth order (thread t examines kItems consecutive ones)
        __syncthreads();
        ushort4 rr[S::kItems];
        uint32_t flags = 0;
#pragma unroll
        for (int k = 0; k < S::kItems; ++k) {
            const int j = jb + S::kItems * threadIdx.x + k;
            rr[k] = j < j1 ? drect[j] : make_ushort4(0, 0, 0, 0);
            bool hit = false;
#pragma unroll
            for (int r = 0; r < kPlaceRows; ++r) {
                const int ty = rb + r;
                hit = hit || (rr[k].y <= ty && ty < rr[k].w && rr[k].x < xhi[r] && rr[k].z > xlo[r]);
            }
            if (rr[k].z > rr[k].x && hit) flags |= 1u << k;
        }
        uint32_t m = 0;
        uint32_t pos = block_exclusive_scan<S::kThreads / 32>((uint32_t)__popc(flags), ws, &m);
#pragma unroll
        for (int k = 0; k < S::kItems; ++k)
            if (flags & (1u << k)) {
                const int j = jb + S::kItems * threadIdx.x + k;
                sr[pos] = rr[k];
                sg[pos] = (uint32_t)dsorted[j];
                sj[pos] = (uint32_t)j;
                ++pos;
            }
        __syncthreads();
        // the tile spans of every (row of the block, compacted Gaussian)
        for (int q = threadIdx.x; q < (int)m; q += S::kThreads) {
            const ushort4 r = sr[q];
            const size_t jj = sj[q];
            const float4 e0 = __ldg(dell + 2 * jj), e1 = __ldg(dell + 2 * jj + 1);
#pragma unroll
            for (int k = 0; k < kPlaceRows; ++k) {
                const int ty = rb + k;
                int xl = 0, xr = 0;
                if (ty < re && r.y <= ty && ty < r.w && r.x < xhi[k] && r.z > xlo[k]) row_span(e0, e1, r, ty, xl, xr);
                span[k][q] = xr > xl ? (uint32_t)xl | ((uint32_t)xr << 16) : 0u;
            }
        }
        __syncthreads();
        if (!row_ok || whi < 0) continue;
        const uint32_t key_hi = (uint32_t)(row * TX + tx);
        for (int q0 = 0; q0 < (int)m; q0 += 32) {
            const uint32_t sp = q0 + lane < (int)m ? span[rloc][q0 + lane] : 0u;
            const uint32_t gl = q0 + lane < (int)m ? sg[q0 + lane] : 0u;
            const int xl = (int)(sp & 0xFFFFu), xr = (int)(sp >> 16);
            uint32_t mask = __ballot_sync(0xffffffffu, xr > xl && xl < whi && xr > wlo);
            if (__popc(mask) > 8 && !keys) {
                // dense: all 32 steps, the spans and ids broadcast from registers (no
                // step waits on the previous one's load)
#pragma unroll
                for (int b = 0; b < 32; ++b) {
                    const uint32_t spb = __shfl_sync(0xffffffffu, sp, b);
                    const uint32_t gid = __shfl_sync(0xffffffffu, gl, b);
                    if (mine && tx >= (int)(spb & 0xFFFFu) && tx < (int)(spb >> 16)) ids[ctr++] = gid;
                }
                continue;
            }
            while (mask) {
                const int b = __ffs(mask) - 1;
                mask &= mask - 1;
                const uint32_t spb = __shfl_sync(0xffffffffu, sp, b);
                const uint32_t gid = __shfl_sync(0xffffffffu, gl, b);
                if (mine && tx >= (int)(spb & 0xFFFFu) && tx < (int)(spb >> 16)) {
                    ids[ctr] = gid;
                    if (keys) keys[ctr] = ((uint64_t)key_hi << 32) | __float_as_uint(depth[gid]);
                    ++ctr;
                }
            }
        }
    }
}

__global__ void ranges_kernel(int T, int nchunks, const uint32_t* __restrict__ base, uint32_t* __restrict__ ranges)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const uint32_t s = base[(size_t)t * nchunks], e = base[(size_t)(t + 1) * nchunks];
    ranges[2 * t] = s == e ? 0u : s;
    ranges[2 * t + 1] = s == e ? 0u : e;
}

// ----------------------------------------------------------------------------
constexpr int kMaxTiles = 16384;

struct SortWs {
    uint64_t *eA, *eB;
    ushort4* drect;
    float4* dell;
    uint32_t *counts, *base, *partials;   // counts: the depth sort's per-tile digit counts / offsets
    uint32_t* sort_state;   // the depth sort's digit totals, [passes][256]
    uint8_t* flags;         // lazy placement: two tile-activity arrays and two row-group arrays, [kMaxTiles] each
    int nchunks, chunk;
    size_t bytes;
};


__host__ __device__ constexpr int chunks_for(int n)
{
    return n <= 0 ? 1 : ((n + 511) / 512 < 1024 ? (n + 511) / 512 : 1024);
}

__host__ __device__ constexpr size_t seg(size_t bytes) { return (bytes + 255) / 256 * 256; }

// The depth sort's digit totals, [passes][256].
__host__ __device__ constexpr size_t sort_state_words(int) { return (size_t)kSortPasses * 256; }

// The depth sort's per-tile counts / offsets, [256][sort_row(n)].
__host__ __device__ constexpr size_t sort_count_words(int n) { return 256ull * sort_row(n); }

// Scratch layout of le_bin_sort for n Gaussians (independent of the copy count).
__host__ __device__ constexpr size_t sort_ws_bytes(int n)
{
    return seg(8ull * n) * 3 + seg(32ull * n) + seg(4ull * sort_count_words(n)) +
           seg(4ull * ((size_t)kMaxTiles * chunks_for(n) + 1)) +
           seg(4ull * (((size_t)kMaxTiles * chunks_for(n) + 1) / kTile + 2)) + seg(4ull * sort_state_words(n)) +
           seg(4ull * kMaxTiles);
}

SortWs sort_ws_layout(char* base, int32_t n)
{
    SortWs w;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += seg(bytes);
        return p;
    };
    w.nchunks = chunks_for(n);
    w.chunk = n > 0 ? (n + w.nchunks - 1) / w.nchunks : 1;
    const size_t count_len = (size_t)kMaxTiles * w.nchunks + 1;
    w.eA = (uint64_t*)take(8ull * n);
    w.eB = (uint64_t*)take(8ull * n);
    w.drect = (ushort4*)take(8ull * n);
    w.dell = (float4*)take(32ull * n);
    w.counts = (uint32_t*)take(4ull * sort_count_words(n));
    w.base = (uint32_t*)take(4ull * count_len);
    w.partials = (uint32_t*)take(4ull * (count_len / kTile + 2));
    w.sort_state = (uint32_t*)take(4ull * sort_state_words(n));
    w.flags = (uint8_t*)take(4ull * kMaxTiles);
    w.bytes = off;
    return w;
}

// The four passes (pass 0's counts are in w.counts and w.sort_state, counted
// by depth_elems_kernel).  Result in *cur; the rectangles and tile ellipses in
// depth order in w.drect and w.dell.
le_status depth_sort(uint64_t*& cur, uint64_t*& alt, int n, const SortWs& w, const int* tiles, const ushort4* rect,
                     const float4* ell, cudaStream_t s)
{
    const int nt = sort_tiles(n), row = sort_row(n);
    for (int q = 0; q < kSortPasses; ++q) {
        const int shift = 32 + 8 * q;
        uint32_t* totals = w.sort_state + 256 * q;
        if (q > 0) {
            sort_count_kernel<<<nt, kSortThreads, 0, s>>>(cur, n, shift, w.counts, row, totals);
            LE_LAUNCHED();
        }
        sort_rowscan_kernel<<<256 / 8, 256, 0, s>>>(w.counts, nt, row, totals);
        LE_LAUNCHED();
        SortGather g{};
        if (q == kSortPasses - 1) g = SortGather{tiles, rect, ell, w.drect, w.dell};
        sort_scatter_kernel<<<nt, kSortThreads, 0, s>>>(cur, alt, n, shift, w.counts, row, g);
        LE_LAUNCHED();
        uint64_t* t = cur;
        cur = alt;
        alt = t;
    }
    return LE_OK;
}

}  // namespace
}  // namespace leg

using namespace leg;

extern "C" le_status le_bin_sort_workspace(int32_t n, int64_t k_cap, size_t* bytes)
{
    LE_TRACE("le_bin_sort_workspace");
    LE_CHECK_ARG(bytes != nullptr, "bytes is null");
    LE_CHECK_ARG(n >= 0 && k_cap >= 0 && k_cap < (int64_t)1 << 31, "n or k_cap out of range");
    *bytes = sort_ws_layout(nullptr, n).bytes;
    return LE_OK;
}

namespace leg {
namespace {

// Steps 1-4 of the binning (depth sort, counts, tile-major scan, K, ranges):
// everything except placing the copies.  Returns with *K = 0 and nothing
// launched beyond the range reset when n == 0.
le_status bin_prepare(const le_camera* cam, int32_t n, const float* depth, const uint16_t* rect,
                      const float* tile_ellipse, const int32_t* tiles_touched, void* workspace,
                      size_t workspace_bytes, int64_t k_cap, bool need_ids, uint32_t* tile_ranges, int64_t* k_out,
                      cudaStream_t s, SortWs& w, uint64_t*& cur)
{
    le_status st = check_camera(cam);
    if (st != LE_OK) return st;
    LE_CHECK_ARG(n >= 0 && k_cap >= 0 && k_cap < (int64_t)1 << 31, "n or k_cap out of range");
    LE_CHECK_ARG(k_out != nullptr && tile_ranges != nullptr, "k_out and tile_ranges are required");
    LE_CHECK_ARG(n == 0 || (depth && rect && tile_ellipse && tiles_touched), "null input pointer");
    LE_CHECK_ARG(k_cap == 0 || need_ids, "sorted_ids is null");
    LE_CHECK_ARG(workspace && (reinterpret_cast<uintptr_t>(workspace) & 255u) == 0,
                 "workspace must be non-null and 256-byte aligned");
    LE_CHECK_ARG((reinterpret_cast<uintptr_t>(rect) & 7u) == 0, "rect must be 8-byte aligned");
    LE_CHECK_ARG((reinterpret_cast<uintptr_t>(tile_ellipse) & 15u) == 0, "tile_ellipse must be 16-byte aligned");
    w = sort_ws_layout(static_cast<char*>(workspace), n);
    LE_CHECK_ARG(workspace_bytes >= w.bytes, "workspace too small: %zu < %zu", workspace_bytes, w.bytes);
    const int TX = tiles_x(cam), TY = tiles_y(cam);
    const int ntiles = TX * TY;
    if (ntiles > kMaxTiles || TX > 256) {
        set_error("%d x %d screen tiles exceed the supported %d tiles / 256 columns", TX, TY, kMaxTiles);
        return LE_ERR_UNSUPPORTED;
    }
    // the ranges are zero unless ranges_kernel writes them all (K > 0)
    const size_t range_bytes = sizeof(uint32_t) * 2 * (size_t)ntiles;
    *k_out = 0;
    if (n == 0) {
        LE_CUDA(cudaMemsetAsync(tile_ranges, 0, range_bytes, s));
        return LE_OK;
    }

    // 1-2: sort the Gaussians by depth (stable: equal depths keep index order; culled last)
    LE_CUDA(cudaMemsetAsync(w.sort_state, 0, 4 * sort_state_words(n), s));
    depth_elems_kernel<<<sort_tiles(n), kSortThreads, 0, s>>>(n, depth, tiles_touched, w.eA, w.counts, sort_row(n),
                                                              w.sort_state);
    LE_LAUNCHED();
    cur = w.eA;
    uint64_t* alt = w.eB;
    // 3: (with the last pass) rectangles and ellipses in depth order
    if ((st = depth_sort(cur, alt, n, w, tiles_touched, reinterpret_cast<const ushort4*>(rect),
                         reinterpret_cast<const float4*>(tile_ellipse), s)) != LE_OK)
        return st;
    // copies per (tile, chunk of depth-sorted Gaussians)
    const size_t diff_smem = sizeof(int4) * (((size_t)(TX + 1) * TY + 3) / 4);
    if (diff_smem > 48 * 1024)
        LE_CUDA(cudaFuncSetAttribute(chunk_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)diff_smem));
    chunk_count_kernel<<<w.nchunks, 512, diff_smem, s>>>(n, w.drect, w.dell, TX, TY, w.chunk, w.nchunks, w.base);
    LE_LAUNCHED();
    // 4: one exclusive scan in tile-major order gives every (tile, chunk) base and K
    const int len = ntiles * w.nchunks;
    if ((st = exclusive_scan(DirectIn{w.base}, len, w.base, w.partials, w.base + len, s)) != LE_OK) return st;
    uint32_t K32 = 0;
    LE_CUDA(cudaMemcpyAsync(&K32, w.base + len, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    LE_CUDA(cudaStreamSynchronize(s));
    *k_out = K32;
    if ((int64_t)K32 > k_cap) {
        LE_CUDA(cudaMemsetAsync(tile_ranges, 0, range_bytes, s));
        set_error("instance count K = %u exceeds k_cap = %lld", K32, (long long)k_cap);
        return LE_ERR_CAPACITY;
    }
    if (K32 == 0) {
        LE_CUDA(cudaMemsetAsync(tile_ranges, 0, range_bytes, s));
        return LE_OK;
    }
    ranges_kernel<<<(ntiles + 255) / 256, 256, 0, s>>>(ntiles, w.nchunks, w.base, tile_ranges);
    LE_LAUNCHED();
    return LE_OK;
}

// Placement geometry: super-chunks of `cs` count chunks, small enough for about
// eight waves of blocks when every chunk is placed (row groups differ a lot in
// work; many short blocks balance them); one chunk each for the lazy phases,
// whose first phase covers only the nearest few chunks.
struct PlaceGrid {
    int ngroups, cs, nsuper, nk;
};

PlaceGrid place_grid(const le_camera* cam, const SortWs& w, bool lazy)
{
    PlaceGrid g;
    const int TY = tiles_y(cam);
    g.ngroups = (TY + kPlaceRows - 1) / kPlaceRows;
    const int want = (8 * 1216 + g.ngroups - 1) / g.ngroups;
    g.cs = !lazy && w.nchunks / want > 1 ? w.nchunks / want : 1;
    g.nsuper = (w.nchunks + g.cs - 1) / g.cs;
    g.nk = (tiles_x(cam) + 31) / 32;
    return g;
}

// Step 5 for super-chunks [s0, s1): place the copies of the active tiles.
le_status place(const le_camera* cam, int32_t n, const float* depth, const SortWs& w, const uint64_t* cur,
                const PlaceGrid& g, int s0, int s1, const uint8_t* tile_act, const uint8_t* rows_act,
                uint32_t* sorted_ids, uint64_t* sorted_keys, cudaStream_t s, uint8_t* zero_a = nullptr,
                int zero_na = 0, uint8_t* zero_r = nullptr, int zero_nr = 0)
{
    if (s1 <= s0) return LE_OK;
    const dim3 grid(g.ngroups, s1 - s0);
    const int TX = tiles_x(cam), TY = tiles_y(cam);
#define LE_PLACE(NS)                                                                                         \
    place_kernel<NS><<<grid, PlaceShape<NS>::kThreads, 0, s>>>(n, cur, w.drect, w.dell, depth, TX, TY,          \
                                                              w.chunk * g.cs, g.cs, w.nchunks, w.base,         \
                                                              sorted_ids, sorted_keys, tile_act, rows_act, s0, zero_a, zero_na,   \
                                                              zero_r, zero_nr)
    switch (g.nk) {
        case 1: LE_PLACE(1); break;
        case 2: LE_PLACE(2); break;
        case 3: LE_PLACE(3); break;
        case 4: LE_PLACE(4); break;
        case 5: LE_PLACE(5); break;
        case 6: LE_PLACE(6); break;
        case 7: LE_PLACE(7); break;
        default: LE_PLACE(8); break;
    }
#undef LE_PLACE
    LE_LAUNCHED();
    return LE_OK;
}

}  // namespace

le_status render_fwd_phase(const le_camera* cam, const float* splat, const uint32_t* ids, const uint32_t* base,
                           int nchunks, int c_lo, int c_hi, const uint8_t* act, uint8_t* next_act,
                           uint8_t* next_rows, float* out_rgb, float* out_feat, float* out_unc, float* T_final,
                           int32_t* n_contrib, cudaStream_t s);
}  // namespace leg

extern "C" le_status le_bin_sort(const le_camera* cam, int32_t n, const float* depth, const uint16_t* rect,
                                 const float* tile_ellipse, const int32_t* tiles_touched, void* workspace,
                                 size_t workspace_bytes, int64_t k_cap,
                                 uint32_t* sorted_ids, uint64_t* sorted_keys, uint32_t* tile_ranges, int64_t* k_out,
                                 void* stream)
{
    LE_TRACE("le_bin_sort");
    cudaStream_t s = as_stream(stream);
    SortWs w;
    uint64_t* cur = nullptr;
    le_status st = bin_prepare(cam, n, depth, rect, tile_ellipse, tiles_touched, workspace, workspace_bytes, k_cap,
                               sorted_ids != nullptr, tile_ranges, k_out, s, w, cur);
    if (st != LE_OK || n == 0 || *k_out == 0) return st;
    const PlaceGrid g = place_grid(cam, w, false);
    return place(cam, n, depth, w, cur, g, 0, g.nsuper, nullptr, nullptr, sorted_ids, sorted_keys, s);
}

extern "C" le_status le_bin_render_fwd(const le_camera* cam, int32_t n, const float* splat, const float* depth,
                                       const uint16_t* rect, const float* tile_ellipse,
                                       const int32_t* tiles_touched, void* workspace, size_t workspace_bytes,
                                       int64_t k_cap, uint32_t* sorted_ids, uint32_t* tile_ranges, int64_t* k_out,
                                       float* out_rgb, float* out_feat, float* out_unc, float* T_final,
                                       int32_t* n_contrib, void* stream)
{
    LE_TRACE("le_bin_render_fwd");
    LE_CHECK_ARG(out_rgb && out_feat && out_unc && T_final && n_contrib, "null output pointer");
    LE_CHECK_ARG(n == 0 || (splat && aligned16(splat)), "splat must be non-null and 16-byte aligned");
    cudaStream_t s = as_stream(stream);
    SortWs w;
    uint64_t* cur = nullptr;
    le_status st = bin_prepare(cam, n, depth, rect, tile_ellipse, tiles_touched, workspace, workspace_bytes, k_cap,
                               sorted_ids != nullptr, tile_ranges, k_out, s, w, cur);
    if (st != LE_OK) return st;
    const int ntiles = tiles_x(cam) * tiles_y(cam);
    if (n == 0 || *k_out == 0) {
        // nothing to place: one render pass over empty lists writes the background
        LE_CUDA(cudaMemsetAsync(w.flags, 0, 4 * kMaxTiles, s));
        if (n == 0) {
            LE_CUDA(cudaMemsetAsync(w.base, 0, sizeof(uint32_t) * ((size_t)ntiles * w.nchunks + 1), s));
        }
        return render_fwd_phase(cam, splat, sorted_ids, w.base, w.nchunks, 0, w.nchunks, nullptr, w.flags,
                                w.flags + 2 * kMaxTiles, out_rgb, out_feat, out_unc, T_final, n_contrib, s);
    }
    // Lazy placement: only 1-2 % of the copies are ever read -- every pixel
    // stops once its transmittance falls below 1e-4, long before the end of its
    // tile's depth-ordered list.  So the depth chunks are placed and rendered
    // in phases [0, 16), [16, 64), [64, 256), [256, all), each phase only for
    // the tiles with a pixel still blending; a tile's later chunks are never
    // written.  The result equals placing everything and rendering once, bit
    // for bit (the same entries are blended in the same order).
    const PlaceGrid g = place_grid(cam, w, true);
    const int bounds[5] = {0, 16, 64, 256, 1 << 30};
    uint8_t* act[2] = {w.flags, w.flags + kMaxTiles};
    uint8_t* rows[2] = {w.flags + 2 * kMaxTiles, w.flags + 3 * kMaxTiles};
    const int ngroups = (tiles_y(cam) + kPlaceRows - 1) / kPlaceRows;
    int lo = 0, phase = 0;
    for (int b = 1; b < 5 && lo < w.nchunks; ++b) {
        int hi = bounds[b] >= w.nchunks ? w.nchunks : (bounds[b] + g.cs - 1) / g.cs * g.cs;
        if (hi > w.nchunks) hi = w.nchunks;
        if (hi <= lo) continue;
        const uint8_t* a = phase == 0 ? nullptr : act[phase & 1];
        const uint8_t* r = phase == 0 ? nullptr : rows[phase & 1];
        uint8_t* na = act[(phase + 1) & 1];
        uint8_t* nr = rows[(phase + 1) & 1];
        const int s0 = lo / g.cs, s1 = (hi + g.cs - 1) / g.cs;
        // the placement also clears na and nr, which this phase's render sets
        if ((st = place(cam, n, depth, w, cur, g, s0, s1, a, r, sorted_ids, nullptr, s, na, ntiles, nr, ngroups)) !=
            LE_OK)
            return st;
        if ((st = render_fwd_phase(cam, splat, sorted_ids, w.base, w.nchunks, lo, hi, a, na, nr, out_rgb, out_feat,
                                   out_unc, T_final, n_contrib, s)) != LE_OK)
            return st;
        lo = hi;
        ++phase;
    }
    return LE_OK;
}

// ----------------------------------------------------------------------------
// le_bin_sort_static: le_bin_sort for callers that cannot allocate device
// memory.  Its scratch is the file-scope array below, sized for at most
// LE_STATIC_MAX_GAUSSIANS Gaussians; every GPU that loads this library holds
// it until the process exits.
namespace leg {
namespace {

constexpr int32_t kStaticMaxN = LE_STATIC_MAX_GAUSSIANS;
constexpr int64_t kStaticMaxK = LE_STATIC_MAX_INSTANCES;

__device__ __align__(256) unsigned char g_static_scratch[sort_ws_bytes(kStaticMaxN)];

// Device address of g_static_scratch in the calling thread's current context.
// It is looked up on every call rather than cached: a cache keyed by device
// would outlive the context (cudaDeviceReset, or another context made current
// on that device) and hand a later call a dangling address.  After the first
// call on a device has loaded this library's module the lookup is a host-side
// table query, small next to the stream synchronisation every call makes.
le_status static_scratch(void** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
        set_error("cudaGetSymbolAddress(static scratch) failed: %s", cudaGetErrorString(e));
        return LE_ERR_CUDA;
    }
    *out = p;
    return LE_OK;
}

}  // namespace
}  // namespace leg

extern "C" le_status le_bin_sort_static(const le_camera* cam, int32_t n, const float* depth, const uint16_t* rect,
                                        const float* tile_ellipse, const int32_t* tiles_touched, int64_t k_cap,
                                        uint32_t* sorted_ids, uint64_t* sorted_keys, uint32_t* tile_ranges,
                                        int64_t* k_out, void* stream)
{
    LE_TRACE("le_bin_sort_static");
    LE_CHECK_ARG(n >= 0 && n <= kStaticMaxN, "n = %d exceeds the static-scratch limit of %d Gaussians", n,
                 kStaticMaxN);
    LE_CHECK_ARG(k_cap >= 0, "k_cap < 0");
    if (k_cap > kStaticMaxK) k_cap = kStaticMaxK;
    size_t need = 0;
    le_status st = le_bin_sort_workspace(n, k_cap, &need);
    if (st != LE_OK) return st;
    if (need > sizeof(g_static_scratch)) {
        set_error("static scratch too small for n = %d", n);
        return LE_ERR_INVALID_ARG;
    }
    void* ws = nullptr;
    if ((st = static_scratch(&ws)) != LE_OK) return st;
    st = le_bin_sort(cam, n, depth, rect, tile_ellipse, tiles_touched, ws, sizeof(g_static_scratch), k_cap,
                     sorted_ids, sorted_keys, tile_ranges, k_out, stream);
    if (st == LE_ERR_CAPACITY && k_out && *k_out > kStaticMaxK)
        set_error("instance count K = %lld exceeds the static-scratch limit of %lld tile copies",
                  (long long)*k_out, (long long)kStaticMaxK);
    return st;
}
