/*
 * Oracle tile binning (integers only).  Test infrastructure only; see oracle.h.
 *
 * The rasterizer the paper reuses (Sec. 4) duplicates every visible Gaussian
 * once per 16x16 tile its rectangle covers, keys each copy with
 *     key = (tile_id << 32) | float_bits(depth),   tile_id = ty * TX + tx
 * (depth > near > 0, so the float bits order like the depths), sorts the keys
 * and cuts the sorted list into one contiguous range per tile.
 *
 * orc_bin writes the keys in emission order (Gaussian index, then the
 * rectangle row by row), sorts them with a stable merge sort -- so equal keys
 * keep emission order, i.e. ties go to the lower Gaussian index (reading) --
 * and writes ranges[tile] = [start, end), empty tiles (0, 0) (reading).
 *
 * orc_tile_list is a brute-force restatement for one tile: scan all Gaussians,
 * keep those whose rectangle contains the tile, order them by (depth, index).
 *
 * Tile ellipse (this implementation's addition; see keypath.c): when `ell` is
 * given, a rectangle row keeps only the tiles of orc_row_span -- those whose
 * pixel-centre box meets the Gaussian's alpha >= 1/255 ellipse, widened by the
 * key path's margins.  The ellipse is convex, so its tiles in one row are
 * contiguous.  For the row band dy in [lo, hi] (pixel centres of the row minus
 * the mean, widened by pady) the band's right-most point of the ellipse is at
 * dy = clamp(ystar, lo, hi) and its left-most at clamp(-ystar, lo, hi), because
 * the right end s dy + sqrt(k (mm - dy^2)) of a row is concave in dy and peaks
 * at ystar (the left end mirrors it).  Evaluated in FP32 in this fixed order,
 * which the GPU binning repeats operation for operation.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static uint32_t fbits(float f)
{
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

/* Tiles [*xl, *xr) of rectangle row ty that meet the tile ellipse E. */
void orc_row_span(const float* E, const int32_t* r, int ty, int* xl, int* xr)
{
    const float mx = E[0], my = E[1], s = E[2], k = E[3], mm = E[4], ystar = E[5], padx = E[6], pady = E[7];
    *xl = *xr = r[0];
    const float yc = (float)(16 * ty) - my;
    const float lo = yc - pady;
    const float hi = (yc + 15.0f) + pady;
    const float dR = fminf(fmaxf(ystar, lo), hi);
    const float dL = fminf(fmaxf(-ystar, lo), hi);
    const float vR = mm - dR * dR;
    const float vL = mm - dL * dL;
    if (!(vR >= 0.0f) || !(vL >= 0.0f)) return;
    const float R = s * dR + sqrtf(k * vR);
    const float L = s * dL - sqrtf(k * vL);
    const float fl = ceilf((((mx + L) - padx) - 15.0f) * 0.0625f);
    const float fr = floorf(((mx + R) + padx) * 0.0625f) + 1.0f;
    const float x0 = (float)r[0], x1 = (float)r[2];
    *xl = (int)fminf(fmaxf(fl, x0), x1);
    *xr = (int)fminf(fmaxf(fr, x0), x1);
    if (*xr < *xl) *xr = *xl;
}

int64_t orc_bin(int N, const orc_cam* cam, const float* depth, const int32_t* rect, const int32_t* tiles,
                const float* ell, uint64_t* keys, uint32_t* vals, uint32_t* ranges)
{
    const int TX = (cam->W + ORC_TILE - 1) / ORC_TILE;
    const int TY = (cam->H + ORC_TILE - 1) / ORC_TILE;
    int64_t K = 0;
    for (int i = 0; i < N; ++i) {
        if (tiles[i] <= 0) continue;
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty) {
            int xl = rect[4 * i], xr = rect[4 * i + 2];
            if (ell) orc_row_span(ell + 8 * (size_t)i, rect + 4 * i, ty, &xl, &xr);
            for (int tx = xl; tx < xr; ++tx) {
                keys[K] = ((uint64_t)(uint32_t)(ty * TX + tx) << 32) | fbits(depth[i]);
                vals[K] = (uint32_t)i;
                ++K;
            }
        }
    }
    /* bottom-up stable merge sort of (key, val) pairs */
    uint64_t* kb = (uint64_t*)malloc(sizeof(uint64_t) * (K > 0 ? K : 1));
    uint32_t* vb = (uint32_t*)malloc(sizeof(uint32_t) * (K > 0 ? K : 1));
    uint64_t *ks = keys, *kd = kb;
    uint32_t *vs = vals, *vd = vb;
    for (int64_t w = 1; w < K; w *= 2) {
        for (int64_t lo = 0; lo < K; lo += 2 * w) {
            int64_t mid = lo + w < K ? lo + w : K;
            int64_t hi = lo + 2 * w < K ? lo + 2 * w : K;
            int64_t i = lo, j = mid, o = lo;
            while (i < mid && j < hi) {
                if (ks[j] < ks[i]) { kd[o] = ks[j]; vd[o++] = vs[j++]; }
                else               { kd[o] = ks[i]; vd[o++] = vs[i++]; }
            }
            while (i < mid) { kd[o] = ks[i]; vd[o++] = vs[i++]; }
            while (j < hi)  { kd[o] = ks[j]; vd[o++] = vs[j++]; }
        }
        uint64_t* tk = ks; ks = kd; kd = tk;
        uint32_t* tv = vs; vs = vd; vd = tv;
    }
    if (ks != keys) {
        memcpy(keys, ks, sizeof(uint64_t) * K);
        memcpy(vals, vs, sizeof(uint32_t) * K);
    }
    free(kb);
    free(vb);
    memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)TX * TY);
    for (int64_t k = 0; k < K; ++k) {
        const uint32_t t = (uint32_t)(keys[k] >> 32);
        if (k == 0 || (uint32_t)(keys[k - 1] >> 32) != t) ranges[2 * t] = (uint32_t)k;
        if (k == K - 1 || (uint32_t)(keys[k + 1] >> 32) != t) ranges[2 * t + 1] = (uint32_t)(k + 1);
    }
    return K;
}

/* Number of copies orc_bin emits (no keys, no sort). */
int64_t orc_bin_count(int N, const int32_t* rect, const int32_t* tiles, const float* ell)
{
    int64_t K = 0;
    for (int i = 0; i < N; ++i) {
        if (tiles[i] <= 0) continue;
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty) {
            int xl = rect[4 * i], xr = rect[4 * i + 2];
            if (ell) orc_row_span(ell + 8 * (size_t)i, rect + 4 * i, ty, &xl, &xr);
            K += xr - xl;
        }
    }
    return K;
}

typedef struct {
    float d;
    uint32_t i;
} depth_idx;

static int cmp_depth_idx(const void* a, const void* b)
{
    const depth_idx* x = (const depth_idx*)a;
    const depth_idx* y = (const depth_idx*)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->i < y->i) ? -1 : (x->i > y->i);
}

int orc_tile_list(int N, const float* depth, const int32_t* rect, const int32_t* tiles, const float* ell,
                  int tx, int ty, uint32_t* out)
{
    depth_idx* buf = (depth_idx*)malloc(sizeof(depth_idx) * (N > 0 ? N : 1));
    int n = 0;
    for (int i = 0; i < N; ++i) {
        if (tiles[i] <= 0) continue;
        if (ty < rect[4 * i + 1] || ty >= rect[4 * i + 3]) continue;
        int xl = rect[4 * i], xr = rect[4 * i + 2];
        if (ell) orc_row_span(ell + 8 * (size_t)i, rect + 4 * i, ty, &xl, &xr);
        if (tx >= xl && tx < xr) {
            buf[n].d = depth[i];
            buf[n].i = (uint32_t)i;
            ++n;
        }
    }
    qsort(buf, n, sizeof(depth_idx), cmp_depth_idx);
    for (int k = 0; k < n; ++k) out[k] = buf[k].i;
    free(buf);
    return n;
}
