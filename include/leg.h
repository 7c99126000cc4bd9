/*
 * leg.h -- C ABI of the GB300 (sm_103a) hot path of Language Embedded 3D
 * Gaussians (arXiv 2311.18482): the tile-based differentiable Gaussian
 * rasterizer carrying RGB, the compact semantic feature s_G and the
 * uncertainty u, its backward pass, the semantic decoder D_MLP with its
 * cross-entropy training step, open-vocabulary relevancy queries and Adam.
 *
 * Conventions for every entry point
 *   - Pointers are DEVICE pointers owned by the caller unless a comment says
 *     "host".  The library never allocates device memory; scratch comes from a
 *     caller workspace whose size a *_workspace call reports.
 *   - `stream` is a cudaStream_t passed as void*; all work is enqueued on it
 *     asynchronously.  Only le_bin_sort synchronizes (once, to read the
 *     instance count K back to the host).
 *   - Every call returns an le_status.  On error nothing is launched (argument
 *     errors) or the CUDA error is reported (LE_ERR_CUDA); le_last_error()
 *     returns a message for the calling thread.  The library never aborts and
 *     never traps on the device.
 *   - Every entry point opens an NVTX range named after itself for the
 *     duration of the call (visible on profiler timelines; free otherwise).
 *   - Arrays are row-major, FP32 unless stated.  Per-Gaussian data is
 *     structure-of-arrays indexed by Gaussian id; images are planar
 *     [channel][H][W]; pixel (i, j) is sampled at integer coordinates.
 *   - 16-byte alignment is required for `splat`, `grad2d`, `sh` and the
 *     decoder weights (torch allocations satisfy it).
 *   - An empty input (n = 0 Gaussians, P = 0 pixels) is valid: the call reads
 *     and writes no per-element array (those pointers may be null), and
 *     fixed-size outputs (losses, gradients of network weights, images) are
 *     written as for no contribution.
 */
#ifndef LEG_H
#define LEG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LE_OK = 0,
    LE_ERR_INVALID_ARG = 1,   /* null/misaligned pointer, bad size */
    LE_ERR_CAPACITY = 2,      /* instance count K exceeds the caller's capacity */
    LE_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed */
    LE_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    LE_ERR_UNSUPPORTED = 5    /* shape not supported by the requested path */
} le_status;

#define LE_TILE 16            /* screen tiles are 16 x 16 pixels */
#define LE_DFEAT 8            /* compact semantic feature width d_s (Sec. 4) */
#define LE_SPLAT_STRIDE 20    /* floats per splat / grad2d record */

/* Pinhole camera, OpenCV axes (x right, y down, z forward).  Host struct.
 * p_cam of Eq. 1 (eq:render): view = world->camera [R | t] (3x4, row-major),
 * campos = camera centre (for the SH view direction). */
typedef struct le_camera {
    float view[12];
    float campos[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_z;             /* Gaussians with view z <= near_z are culled (3DGS: 0.2) */
    float bg[3];              /* background colour; feature / uncertainty backgrounds are 0 */
} le_camera;

/* The 3D Gaussians G (Sec. 3.1: position p, covariance Sigma via scale and
 * rotation, colour c via SH, opacity alpha; Sec. 3.4: semantic feature s_G in
 * R^8 and uncertainty u).  Host struct of device pointers. */
typedef struct le_gaussians {
    int32_t n;
    int32_t sh_degree;        /* 0..3; sh has (sh_degree+1)^2 coefficients per channel */
    const float* means;       /* [n,3] */
    const float* log_scales;  /* [n,3]  scale = exp(log_scale) */
    const float* quats;       /* [n,4]  (w,x,y,z), normalised inside */
    const float* opacity_raw; /* [n]    opacity = sigmoid(opacity_raw) */
    const float* sh;          /* [n,(deg+1)^2,3], coefficient k = l^2+l+m, m=-l..l */
    const float* feat;        /* [n,8]  s_G */
    const float* unc;         /* [n]    u */
} le_gaussians;

/* Gradients with the same shapes as le_gaussians.  Host struct of device pointers. */
typedef struct le_gaussian_grads {
    float* means;
    float* log_scales;
    float* quats;
    float* opacity_raw;
    float* sh;
    float* feat;
    float* unc;
} le_gaussian_grads;

/* Screen-space state produced by le_preprocess.  Host struct of device pointers.
 * splat record, 20 floats per Gaussian (80 bytes, the unit the renderer reads):
 *   [0,1] mean2d x,y  [2,3,4] the conic (A, B, C) = inverse 2D covariance, stored
 *   in base-2 exponent units as (A log2(e)/2, B log2(e), C log2(e)/2), so that
 *   alpha = o 2^-(A' dx^2 + B' dx dy + C' dy^2)  [5] opacity  [6,7,8] rgb  [9] u
 *   [10..17] s_G  [18,19] unused
 * grad2d records (le_render_bwd) use the same layout for dL/d of each field,
 * the conic slots holding dL/dA, dL/dB, dL/dC of the unscaled conic. */
typedef struct le_projected {
    float* splat;             /* [n,20] */
    float* depth;             /* [n]  view-space z (sort key) */
    int32_t* radius;          /* [n]  0 = culled */
    uint16_t* rect;           /* [n,4] tile rectangle x0,y0,x1,y1 (half-open) */
    int32_t* tiles_touched;   /* [n]  (x1-x0)(y1-y0), 0 = culled */
    uint8_t* clamp_mask;      /* [n]  bit c set when colour channel c was clamped at 0 */
    float* tile_ellipse;      /* [n,8] tile ellipse for binning (see le_preprocess), 16-byte aligned */
} le_projected;

/* ---------------------------------------------------------------------------
 * le_preprocess -- project every Gaussian (Eq. 1 (eq:render); the 3DGS
 * projection that Sec. 4 says the method reuses):
 *   Sigma = R S S^T R^T, t = R_c p + t_c, J = d(pinhole)/dt with t_x/t_z,
 *   t_y/t_z clamped to +-1.3 (W/2)/f inside J, Sigma2 = J R_c Sigma R_c^T J^T
 *   + 0.3 I, conic = Sigma2^-1, radius = ceil(3 sqrt(lambda_max)), tile rect,
 *   rgb = max(0, SH(dir) + 0.5).
 * Depth, screen mean, Sigma2, radius and rect are computed by a fixed
 * sequence of IEEE FP32 operations (explicit FMA chains, exp by Cody-Waite
 * reduction + degree-7 Taylor) so that binning is reproducible bit for bit.
 * The same fixed sequence writes tile_ellipse, which is not in the paper: a
 * conservative form of the ellipse where o exp(-q/2) >= 1/255, used by
 * le_bin_sort to skip the rect tiles no pixel of which the Gaussian can
 * reach.  With Sigma2 = [[a,b],[b,c]], t = (2 lnu(255 o) + 1/16)(1 + 2^-10)
 * (lnu an upper bound of ln from the exponent and (m-1)/sqrt(m)), r the
 * radius: {mx, my, b/c, det/c^2, c t, b sqrt(t/a), 1/4 + 2^-12(|mx| + 2r),
 * 1/4 + 2^-12(|my| + 2r)} (c t = -1 when t <= 0).
 * tiles_touched is the rect's tile count, an upper bound of the copies.
 * Culled Gaussians get radius = tiles_touched = 0 and a zero splat record.
 * Errors: LE_ERR_INVALID_ARG for n < 0, sh_degree outside 0..3, null or
 * misaligned pointers. */
le_status le_preprocess(const le_gaussians* g, const le_camera* cam, le_projected* out, void* stream);

/* ---------------------------------------------------------------------------
 * le_bin_sort -- duplicate each visible Gaussian once per tile of its rect
 * that its tile ellipse reaches, key each copy (tile_id << 32) |
 * float_bits(depth), tile_id = ty*TX + tx, order the copies by key with ties
 * kept in emission order (Gaussian index), and cut the order into per-tile
 * ranges (the 3DGS binning of Sec. 4; tie rule and empty range (0,0) are
 * readings).  Tile ellipse (not in the paper; see le_preprocess): in rect row
 * ty, with lo/hi = 16 ty (+15) - my -/+ pady, dR = clamp(ystar, lo, hi), dL =
 * clamp(-ystar, lo, hi), the row keeps tiles [ceil((mx + s dL - sqrt(k (mm -
 * dL^2)) - padx - 15)/16), floor((mx + s dR + sqrt(k (mm - dR^2)) + padx)/16)
 * + 1) clipped to the rect, none if mm < dR^2 or mm < dL^2; the left-out
 * tiles hold no pixel where the renderer's alpha reaches 1/255, so images and
 * gradients equal those of whole-rect binning.  The K copies are never sorted:
 * the Gaussians are radix-sorted by depth, per-(tile, chunk-of-Gaussians)
 * copy counts come from per-row difference arrays of those spans, one
 * exclusive scan of the counts in tile-major order gives every chunk's offset
 * inside every tile's range, and each chunk writes its copies in depth order
 * -- the same order as a stable sort of the full keys.
 *   depth, rect, tile_ellipse, tiles_touched: from le_preprocess (n entries)
 *   workspace: le_bin_sort_workspace(n, k_cap) bytes, 256-byte aligned (it
 *     depends on n only; k_cap bounds the outputs)
 *   sorted_ids:  [k_cap] out, Gaussian id of each copy in key order
 *   sorted_keys: [k_cap] out, nullable; the 64-bit keys in order
 *   tile_ranges: [TX*TY, 2] out, [start, end) into sorted_ids
 *   k_out: HOST pointer, receives K (always, also on LE_ERR_CAPACITY)
 * Synchronizes `stream` once to read K.  LE_ERR_CAPACITY when K > k_cap
 * (nothing after the count is launched; retry with k_cap >= *k_out).
 * LE_ERR_UNSUPPORTED for more than 16384 screen tiles or 256 tile columns. */
le_status le_bin_sort_workspace(int32_t n, int64_t k_cap, size_t* bytes);
le_status le_bin_sort(const le_camera* cam, int32_t n, const float* depth, const uint16_t* rect,
                      const float* tile_ellipse, const int32_t* tiles_touched, void* workspace,
                      size_t workspace_bytes, int64_t k_cap,
                      uint32_t* sorted_ids, uint64_t* sorted_keys, uint32_t* tile_ranges, int64_t* k_out,
                      void* stream);

/* ---------------------------------------------------------------------------
 * le_bin_sort_static -- le_bin_sort without a caller workspace.  (No
 * counterpart in the paper: it is a deployment convenience of this library.)
 * For callers that must not allocate device memory -- for example code that
 * runs inside a host application or plugin whose device memory is owned and
 * budgeted by someone else, or a per-frame path where the implicit
 * synchronisation of cudaMalloc/cudaFree is not acceptable.  It calls no
 * cudaMalloc, cudaFree or other allocating routine; its scratch is a
 * statically sized device array inside this library (about 11.5 MB), which
 * every GPU that loads the library holds until the process exits.
 *   Limits: n <= LE_STATIC_MAX_GAUSSIANS, and at most LE_STATIC_MAX_INSTANCES
 *   tile copies (k_cap is clamped to it).  Larger n -> LE_ERR_INVALID_ARG;
 *   more copies -> LE_ERR_CAPACITY with *k_out = K and a message naming the
 *   limit.  Inputs and outputs are those of le_bin_sort.
 *   Every call looks up the array's device address in the calling thread's
 *   current context (the first call on a device also loads this library's
 *   module there), so a call made after cudaDeviceReset, or with another
 *   context current, uses that context's array.  Like le_bin_sort, it
 *   synchronizes `stream` once to read K.
 *   All calls share the one array, which keeps the last call's contents (every
 *   scratch word is rewritten before it is read, so nothing needs clearing):
 *   calls whose GPU work overlaps -- on different streams or host threads --
 *   race on it and must be serialised by the caller. */
#define LE_STATIC_MAX_GAUSSIANS 65536
#define LE_STATIC_MAX_INSTANCES 524288
le_status le_bin_sort_static(const le_camera* cam, int32_t n, const float* depth, const uint16_t* rect,
                             const float* tile_ellipse, const int32_t* tiles_touched, int64_t k_cap,
                             uint32_t* sorted_ids, uint64_t* sorted_keys, uint32_t* tile_ranges, int64_t* k_out,
                             void* stream);

/* ---------------------------------------------------------------------------
 * le_bin_render_fwd -- le_bin_sort followed by le_render_fwd, with lazy
 * placement (not in the paper; an implementation choice with identical
 * results).  Every pixel stops blending once its transmittance would fall
 * below 1e-4, so only a small front part of each tile's depth-ordered list is
 * ever read (about 1-2 % of the copies at 1M Gaussians).  The depth chunks of
 * the binning (about 1000 depth-consecutive Gaussians each) are placed and
 * rendered in phases -- chunks [0,16), [16,64), [64,256), [256,all) -- each
 * phase only for the tiles that still have a pixel blending; the render of a
 * phase resumes from the state the previous phase left in the outputs.
 *   Inputs: as le_bin_sort, plus splat (from le_preprocess, 16-byte aligned).
 *   Outputs: tile_ranges, *k_out, and the images of le_render_fwd, equal bit
 *   for bit to le_bin_sort + le_render_fwd.  sorted_ids holds every entry that
 *   any pixel of its tile reaches (position < n_contrib) -- everything
 *   le_render_bwd reads; the entries behind the last stopped pixel of a tile
 *   are not written.  No keys are produced.
 *   workspace: le_bin_sort_workspace(n, k_cap) bytes.
 * Synchronizes `stream` once (to read K), as le_bin_sort.  Errors: those of
 * le_bin_sort and le_render_fwd. */
le_status le_bin_render_fwd(const le_camera* cam, int32_t n, const float* splat, const float* depth,
                            const uint16_t* rect, const float* tile_ellipse, const int32_t* tiles_touched,
                            void* workspace, size_t workspace_bytes, int64_t k_cap, uint32_t* sorted_ids,
                            uint32_t* tile_ranges, int64_t* k_out, float* out_rgb, float* out_feat, float* out_unc,
                            float* T_final, int32_t* n_contrib, void* stream);

/* ---------------------------------------------------------------------------
 * le_render_fwd -- per pixel, front to back over its tile's range:
 *   power = -(A dx^2 + C dy^2)/2 - B dx dy (d = mean2d - pixel), skip if > 0;
 *   alpha = min(0.99, o e^power), skip if alpha < 1/255; stop before the
 *   Gaussian that would make T (1 - alpha) < 1e-4;
 *   C += f alpha T for rgb (Eq. 1), s_G (R_s, Sec. 3.4.1), u (R_u, Sec. 3.4.2);
 *   T <- T (1 - alpha); finally rgb += T bg.
 *   out_rgb [3,H,W], out_feat [8,H,W], out_unc [H,W], T_final [H,W],
 *   n_contrib [H,W] = 1 + range position of the last blended Gaussian (0 if none).
 * Errors: LE_ERR_INVALID_ARG for null pointers or bad camera size. */
le_status le_render_fwd(const le_camera* cam, int32_t n, const float* splat, const uint32_t* sorted_ids,
                        const uint32_t* tile_ranges, float* out_rgb, float* out_feat, float* out_unc,
                        float* T_final, int32_t* n_contrib, void* stream);

/* ---------------------------------------------------------------------------
 * le_render_bwd -- gradient of a loss L through le_render_fwd and
 * le_preprocess ("differentiable rendering and gradient descent", Sec. 3.1).
 * Each tile is walked back to front, recomputing the per-pixel transmittance
 * from T_final by division (no per-Gaussian state is stored); per-Gaussian
 * contributions are reduced across each warp before one atomic add per warp.
 *   dL_drgb [3,H,W], dL_dfeat [8,H,W], dL_dunc [H,W]: upstream gradients
 *   grad2d [n,20]: out (caller memory, zeroed by the call), dL/d of the splat
 *                  record fields (screen-space gradients)
 *   out: dL/d of every Gaussian parameter (overwritten, not accumulated).
 * Derivatives of branches are those of the branch taken (alpha clamp at 0.99,
 * guard-band clamp, colour clamp).  Errors: LE_ERR_INVALID_ARG. */
le_status le_render_bwd(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                        const uint32_t* sorted_ids, const uint32_t* tile_ranges, const float* T_final,
                        const int32_t* n_contrib, const float* dL_drgb, const float* dL_dfeat,
                        const float* dL_dunc, float* grad2d, const le_gaussian_grads* out, void* stream);

/* ---------------------------------------------------------------------------
 * le_render_bwd_adam -- le_render_bwd fused with the Adam step of Sec. 4 on
 * the Gaussian parameters: the gradient of each parameter is applied where it
 * is computed and never written to memory.  The arrays of g are updated in
 * place (they must be writable device memory); m and v are the first and
 * second moments, one array per field in the parameters' own layout; u is
 * clamped to [0, 1] (Sec. 3.4.2), the other fields are not clamped.  The
 * result equals le_render_bwd followed by le_adam on every field with the
 * same hyperparameters, bit for bit.
 *   adam: step >= 1 (bias corrections 1 - beta^step), lr, beta1, beta2, eps
 * Errors: LE_ERR_INVALID_ARG (null/misaligned pointers, step < 1). */
typedef struct le_adam_config {
    int32_t step;
    float lr, beta1, beta2, eps;
} le_adam_config;

le_status le_render_bwd_adam(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                             const uint32_t* sorted_ids, const uint32_t* tile_ranges, const float* T_final,
                             const int32_t* n_contrib, const float* dL_drgb, const float* dL_dfeat,
                             const float* dL_dunc, float* grad2d, const le_gaussian_grads* m,
                             const le_gaussian_grads* v, const le_adam_config* adam, void* stream);

/* ---------------------------------------------------------------------------
 * The two halves of le_render_bwd / le_render_bwd_adam as separate calls
 * (same arguments, same results bit for bit), so that a caller can schedule
 * or time them apart:
 * le_render_bwd_screen -- the screen-space half: zeroes grad2d and fills it
 *   with dL/d of every splat record field (the per-pixel back-to-front walk).
 * le_project_bwd -- the projection half: chains grad2d to every Gaussian
 *   parameter through le_preprocess (out: overwritten).
 * le_project_bwd_adam -- the projection half with the Adam step applied where
 *   each gradient is computed (g updated in place, u clamped to [0, 1]), as in
 *   le_render_bwd_adam.
 * grad2d: [n,20], 16-byte aligned, written by le_render_bwd_screen (or by the
 * caller) and only read by the projection half.  Errors: LE_ERR_INVALID_ARG. */
le_status le_render_bwd_screen(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                               const uint32_t* sorted_ids, const uint32_t* tile_ranges, const float* T_final,
                               const int32_t* n_contrib, const float* dL_drgb, const float* dL_dfeat,
                               const float* dL_dunc, float* grad2d, void* stream);
le_status le_project_bwd(const le_camera* cam, const le_gaussians* g, const le_projected* pr, const float* grad2d,
                         const le_gaussian_grads* out, void* stream);
le_status le_project_bwd_adam(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                              const float* grad2d, const le_gaussian_grads* m, const le_gaussian_grads* v,
                              const le_adam_config* adam, void* stream);

/* le_project_bwd_adam_extra -- le_project_bwd_adam that, in the same launch,
 * also applies the same Adam step (Sec. 4; same step, lr, betas and eps; no
 * clamp) to one more flat FP32 range: extra_param (in/out), extra_grad (in),
 * extra_m, extra_v (in/out), n_extra elements each, every pointer 16-byte
 * aligned -- e.g. the decoder parameters whose gradients le_decode wrote.  Per
 * element the same operations as le_adam, so the range ends bit for bit as
 * le_adam would leave it.  n_extra = 0: exactly le_project_bwd_adam.  g->n = 0
 * with n_extra > 0 updates the range only.  Errors: LE_ERR_INVALID_ARG (as
 * le_project_bwd_adam; n_extra < 0; a null or unaligned extra pointer). */
le_status le_project_bwd_adam_extra(const le_camera* cam, const le_gaussians* g, const le_projected* pr,
                                    const float* grad2d, const le_gaussian_grads* m, const le_gaussian_grads* v,
                                    const le_adam_config* adam, float* extra_param, const float* extra_grad,
                                    float* extra_m, float* extra_v, int64_t n_extra, void* stream);

/* ---------------------------------------------------------------------------
 * Semantic decoder D_MLP (Eq. 8, eq:lem_dec; supp. Tab. dmlp): per-pixel MLP
 * d_in(=8) -> h1 -> h2 -> n_cb, ReLU, ReLU, linear.  FP32 device weights
 * [out][in] row-major (a 1x1 convolution's weight), 16-byte aligned. */
typedef struct le_decoder {
    int32_t d_in, h1, h2, n_cb;
    const float *W1, *b1, *W2, *b2, *W3, *b3;
} le_decoder;

typedef struct le_decoder_grads {
    float *W1, *b1, *W2, *b2, *W3, *b3;   /* overwritten */
} le_decoder_grads;

#define LE_DECODE_UNFUSED_FP32 0   /* FP32 CUDA cores, activations and logits through HBM */
#define LE_DECODE_FUSED_BF16 1     /* tcgen05 BF16 tensor cores, FP32 accumulation in TMEM,
                                      logits never leave the chip */

/* le_decode -- inference (target == NULL) or training step (target != NULL).
 *   feat [8,P] = R_s, unc [P] = R_u (training only)
 *   inference outputs (each nullable): argmax [P] (ties -> lowest id),
 *     prob [n_cb,P] = softmax (M_infer, supp. Sec. "Inference"),
 *     logits [n_cb,P] (unfused path only)
 *   training (Eqs. 9-12): loss [2] = (L_CE, L_u) with
 *     L_CE = sum CE_px (1 - u_px)/P, L_u = sum u_px / P (overwritten);
 *     d_feat [8,P], d_unc [P], dgrads = gradient of
 *     L_s = lambda_ce L_CE + lambda_u L_u (u is differentiated too).
 *   workspace: le_decode_workspace bytes (256-byte aligned), queried with
 *     mode | LE_DECODE_TRAIN for a training call.
 * Fused path: d_in = 8 with h1 = 64, h2 = 128 (the two-hidden-layer network
 * at half the widths of supp. Tab. dmlp) or h1 = 128, h2 = 256 (the widths of
 * supp. Tab. dmlp itself), n_cb in {16..256, multiple of 16}, training n_cb <=
 * 128; otherwise LE_ERR_UNSUPPORTED.  At 8-128-256-N a training call needs a
 * workspace of about 1.8 KB per pixel (each 128-pixel tile's BF16 activations
 * and their gradients, written by a first pass and contracted into the weight
 * gradients by a second); inference needs only the weights' images. */
#define LE_DECODE_TRAIN 4           /* le_decode_workspace only: size for a training call */
le_status le_decode_workspace(int32_t mode, int32_t P, const le_decoder* dec, size_t* bytes);
le_status le_decode(int32_t mode, int32_t P, const float* feat, const float* unc, const le_decoder* dec,
                    const int32_t* target, float lambda_ce, float lambda_u, float* loss, float* d_feat,
                    float* d_unc, const le_decoder_grads* dgrads, int32_t* argmax, float* prob, float* logits,
                    void* workspace, size_t workspace_bytes, void* stream);

/* le_decode_l1 -- a le_decode training call that also computes the RGB L1 term
 * of Sec. 4 (le_rgb_l1) over the same P pixels: img, img_target [3,P] (the
 * rendered colour and its target), loss_l1 [1] = mean |img - img_target| over
 * the 3P values (overwritten), d_img [3,P] = sign(img - img_target) / (3P).
 * The other arguments and outputs are le_decode's (training only; target
 * non-null, P > 0).  With LE_DECODE_FUSED_BF16 at 8-64-128-N the tensor-core
 * training kernel computes the L1 term in the same pass (no separate launch);
 * otherwise it is le_rgb_l1 followed by le_decode.  d_img equals le_rgb_l1's
 * bit for bit; loss_l1 matches it up to the order of its FP32 sums.
 * Errors: those of le_decode and le_rgb_l1; a null L1 pointer. */
le_status le_decode_l1(int32_t mode, int32_t P, const float* feat, const float* unc, const le_decoder* dec,
                       const int32_t* target, float lambda_ce, float lambda_u, float* loss, float* d_feat,
                       float* d_unc, const le_decoder_grads* dgrads, const float* img, const float* img_target,
                       float* loss_l1, float* d_img, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * le_query -- relevancy of the language feature map F = M_infer S against
 * text prompts (supp. Sec. "Inference"; relevancy "in accordance with LERF",
 * reading: phi = F_clip/|F_clip|, rel_j = min_k e^{phi.q_j}/(e^{phi.q_j} +
 * e^{phi.n_k}), temperature 1; F_clip = first d_clip dims of F).
 *   codebook S [n_cb,d], text [Q,d_clip], negs [n_neg,d_clip], relevancy [Q,P].
 *   mode LE_DECODE_UNFUSED_FP32: prob [n_cb,P] given (from le_decode);
 *     F is materialised in FP32 chunks through the workspace.
 *   mode LE_DECODE_FUSED_BF16: feat [8,P] + dec given; decode, softmax and
 *     relevancy in one tcgen05 kernel using |F_clip|^2 = p^T (S_c S_c^T) p and
 *     phi.q = p.(S_c q) / |F_clip| (never forms F).
 * dec is required in both modes (its n_cb is the codebook size).  Q >= 1,
 * n_neg >= 1, Q + n_neg <= 16. */
le_status le_query_workspace(int32_t mode, int32_t P, int32_t n_cb, int32_t d_clip, size_t* bytes);
le_status le_query(int32_t mode, int32_t P, const float* feat, const le_decoder* dec, const float* prob,
                   const float* codebook, int32_t d, int32_t d_clip, const float* text, int32_t Q,
                   const float* negs, int32_t n_neg, float* relevancy, void* workspace, size_t workspace_bytes,
                   void* stream);

/* ---------------------------------------------------------------------------
 * le_feature_map -- the language feature map F = M_infer S (supp. Sec.
 * "Inference": M_infer = softmax(D_MLP(R_s)), S the [n_cb, d] codebook),
 * materialised for consumers other than the relevancy query.
 *   feat [8,P] = R_s; dec: the decoder (fused-path sizes, see le_decode);
 *   codebook [n_cb, d] FP32; out [P, d] BF16 (bit patterns), pixel-major,
 *   16-byte aligned; workspace: le_feature_map_workspace(n_cb, d) bytes.
 * One tcgen05 kernel: decode, softmax (stored in BF16, normalised in FP32 at
 * the output), F = p S with FP32 accumulation, BF16 out through TMA tensor
 * stores.  The workspace holds BF16 images of the codebook and of W3.
 * Errors: LE_ERR_INVALID_ARG; LE_ERR_UNSUPPORTED unless d is a multiple of
 * 64 and the decoder has the fused path's sizes. */
le_status le_feature_map_workspace(int32_t n_cb, int32_t d, size_t* bytes);
le_status le_feature_map(int32_t P, const float* feat, const le_decoder* dec, const float* codebook, int32_t d,
                         uint16_t* out, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * le_quantize -- quantisation of K language features against an N-entry
 * codebook (Sec. 3.3, Eqs. eq:quant, eq:q_dist, eq:q_loss_cos, eq:q_loss_lb,
 * eq:q_loss_cb; supplementary "Load Balancing Loss"):
 *   D_ij = cos(F_i^C, f_j^C) + lambda_D cos(F_i^D, f_j^D)
 *     (C = dims [0, d_clip) of the hybrid CLIP+DINO feature, D = the rest)
 *   indices[i] = m_i = argmax_j D_ij (ties -> lowest j): the semantic index map
 *   L_cos = mean_i (1 - cos^C(F_i, f_m)) + lambda_D (1 - cos^D(F_i, f_m))
 *   r = histogram of m / K (utilisation), p = mean_i softmax_j(D_ij)
 *   L_lb = sum_j r_j p_j,  L_q = lambda_cos L_cos + lambda_lb L_lb
 * (the paper: lambda_D = lambda_lb = 0.5, lambda_cos = 1).
 *   features: [K, d] BF16 bit patterns, row-major, 16-byte aligned
 *   codebook: [n_cb, d] FP32; the distances use its BF16 rounding (nearest
 *             even) and the norms of the rounded parts
 *   indices [K] out; r, p [n_cb] out (nullable); loss [3] out = (L_q, L_cos, L_lb)
 *   workspace: le_quantize_workspace(n_cb, d) bytes, 256-byte aligned.
 * Features and codes must have nonzero CLIP and DINO parts.  BF16 operands on
 * the tensor cores, FP32 accumulation, norms, softmax and sums in FP32.
 * Errors: LE_ERR_INVALID_ARG (null/misaligned pointers, K < 1, K >= 2^31,
 * 0 < d_clip < d violated); LE_ERR_UNSUPPORTED unless d and d_clip are
 * multiples of 64 and n_cb is a multiple of 16 in 16..128. */
le_status le_quantize_workspace(int32_t n_cb, int32_t d, size_t* bytes);
le_status le_quantize(int64_t K, int32_t d, int32_t d_clip, const uint16_t* features, int32_t n_cb,
                      const float* codebook, float lambda_d, float lambda_cos, float lambda_lb, int32_t* indices,
                      float* r, float* p, float* loss, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * le_quantize_grad -- gradient of L_q (as le_quantize computes it) with
 * respect to the codebook, for its optimisation (Sec. 3.3, "Optimization"):
 *   g_ij = dL_q/dD_ij = lambda_lb/K s_ij (r_j - sum_k s_ik r_k) - lambda_cos/K [j = m_i]
 *     (s = row softmax of D, r = the utilisation ratio le_quantize returned,
 *      held constant: argmax counts have no derivative)
 *   dL/df_j^C = (sum_i g_ij (F_i^C/|F_i^C| - cos^C_ij f_j^C/|f_j^C|)) / |f_j^C|, and the
 *   same for the DINO part times lambda_D -- with respect to the BF16-rounded
 *   codebook values the distances use.
 *   features, codebook, d, d_clip, n_cb, lambdas: as le_quantize (same values)
 *   r: [n_cb] from le_quantize on the same inputs
 *   grad_codebook: [n_cb, d] FP32 out (overwritten)
 *   workspace: le_quantize_grad_workspace(K, n_cb, d) bytes (it holds the
 *     BF16 matrix g / |F| twice, 4 n_cb K bytes), 256-byte aligned.
 * The contraction over the K features runs on the tensor cores with g
 * rounded to BF16 (about 2^-9 relative per term), FP32 accumulation.
 * Errors: those of le_quantize, and LE_ERR_UNSUPPORTED unless d and d_clip
 * are multiples of 128. */
le_status le_quantize_grad_workspace(int64_t K, int32_t n_cb, int32_t d, size_t* bytes);
le_status le_quantize_grad(int64_t K, int32_t d, int32_t d_clip, const uint16_t* features, int32_t n_cb,
                           const float* codebook, const float* r, float lambda_d, float lambda_cos, float lambda_lb,
                           float* grad_codebook, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Adaptive spatial smoothing (Sec. 3.4, Eqs. eq:lem_fmlp, eq:lem_loss_mlp;
 * supplementary Tab. pemlp): s_MLP = MLP(PE(p)) per Gaussian, PE of frequency
 * 0 (the position itself), MLP 3 -> 128 -> 128 -> 128 -> 8 with ReLU after
 * the first three layers.  FP32 device weights [out][in], biases [out]. */
typedef struct le_smooth_mlp {
    const float *W1, *b1;     /* [128,3], [128] */
    const float *W2, *b2;     /* [128,128], [128] */
    const float *W3, *b3;     /* [128,128], [128] */
    const float *W4, *b4;     /* [8,128], [8] */
} le_smooth_mlp;

typedef struct le_smooth_mlp_grads {
    float *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;   /* same shapes; overwritten */
} le_smooth_mlp_grads;

/* le_smooth -- L_smo = lambda_smo mean_i (|s_MLP - s_G*| + max(u*, w_s) |s_MLP* - s_G|)
 * (* = stop gradient; |.| the plain L2 norm, gradient 0 at a zero difference;
 * the paper's w_s = 0.1, lambda_smo = 1) and its gradients:
 *   loss [1] out (overwritten);
 *   d_feat: dL/ds_G ADDED to d_feat[i * d_feat_stride + c] (c < 8), so that it
 *     can accumulate into a dense [n,8] array (stride 8) or into the feature
 *     slots of le_render_bwd_screen's grad2d records (grad2d + 10, stride 20)
 *     before le_project_bwd_adam applies it;
 *   dmlp: the MLP parameter gradients (overwritten);
 *   s_mlp: [n,8] out, nullable.
 * No gradient reaches the positions or u.  Tensor cores: BF16 operands
 * (positions, weights, activations and dL/ds_MLP rounded to BF16), FP32
 * accumulation; loss, norms and d_feat in FP32.
 * Errors: LE_ERR_INVALID_ARG (null pointers, n < 0, d_feat_stride < 8, feat
 * not 16-byte aligned). */
le_status le_smooth(int32_t n, const float* means, const float* feat, const float* unc, const le_smooth_mlp* mlp,
                    float w_s, float lambda_smo, float* loss, float* d_feat, int32_t d_feat_stride,
                    const le_smooth_mlp_grads* dmlp, float* s_mlp, void* stream);

/* ---------------------------------------------------------------------------
 * Adaptive density control of 3D Gaussian Splatting, which Sec. 4 keeps
 * ("enables adaptive density control of 3D Gaussians during the
 * reconstruction"; reading: 3DGS's clone / split / prune rule).
 * le_densify_stats -- every step after le_render_bwd_screen: for every
 *   Gaussian with radius > 0, acc[i] += sqrt(gx^2 + gy^2) (gx, gy = grad2d
 *   [i][0..1], dL/dmean2d in pixels), cnt[i] += 1, and, when max_radius is
 *   not null, max_radius[i] = max(max_radius[i], radius[i]) (the largest
 *   screen radius since the caller last zeroed the statistics).
 * le_opacity_reset -- 3DGS's periodic opacity reset: opacity_raw[i] =
 *   min(opacity_raw[i], fl(logit(max_opacity))) (opacity = min(opacity,
 *   max_opacity); 3DGS: 0.01) and the opacity's Adam moments m, v zeroed.
 *   n floats each, device pointers.  LE_ERR_INVALID_ARG for max_opacity
 *   outside (0, 1).
 * le_densify -- with g_i = acc_i / cnt_i: pruned if sigmoid(opacity_raw) <
 *   min_opacity, or (size pruning, 3DGS's removal of Gaussians too large in
 *   view and world space) if max_screen_size > 0 and max_radius_i >
 *   max_screen_size, or if world_frac > 0 and its largest scale > world_frac *
 *   scene_extent; a pruned Gaussian is neither cloned nor split (max_radius
 *   may be null when max_screen_size == 0); else split if g_i >= grad_thresh
 *   and its largest scale >
 *   percent_dense * scene_extent; else cloned if g_i >= grad_thresh; else kept.
 *   The decisions are FP32 comparisons against thresholds computed in double
 *   (opacity_raw < logit(min_opacity), max log-scale > ln(percent_dense *
 *   extent), max log-scale > ln(world_frac * extent), (float)max_radius >
 *   max_screen_size, cnt > 0 and acc >= fl(grad_thresh * cnt)), reproducible
 *   bit for bit.
 *   Output (g_out, m_out, v_out, capacity n_cap Gaussians each): the kept and
 *   cloned Gaussians in index order, then the clones, then two children per
 *   split Gaussian; a child k copies its parent except mean = mu + R(q)
 *   diag(exp(log-scale)) noise[i][k] and log-scale - ln(1.6).  Adam moments
 *   are carried for kept Gaussians and zero for clones and children.
 *   noise: [n,2,3] standard normal samples (the caller draws them).
 *   n_out: HOST pointer, the output count (also on LE_ERR_CAPACITY).
 *   workspace: le_densify_workspace(n) bytes.  Synchronizes `stream` once.
 * Errors: LE_ERR_INVALID_ARG; LE_ERR_CAPACITY when the output exceeds n_cap. */
typedef struct le_densify_config {
    float grad_thresh;       /* mean |dL/dmean2d| in pixels */
    float percent_dense;     /* 3DGS: 0.01 */
    float scene_extent;
    float min_opacity;       /* 3DGS: 0.005 */
    float max_screen_size;   /* pixels; 0 = off (3DGS: 20 once opacity resets have begun) */
    float world_frac;        /* fraction of scene_extent; 0 = off (3DGS: 0.1, with the screen test) */
} le_densify_config;

le_status le_densify_stats(int32_t n, const float* grad2d, const int32_t* radius, float* acc, int32_t* cnt,
                           int32_t* max_radius, void* stream);
le_status le_opacity_reset(int32_t n, float* opacity_raw, float* m_opacity, float* v_opacity, float max_opacity,
                           void* stream);
le_status le_densify_workspace(int32_t n, size_t* bytes);
le_status le_densify(const le_densify_config* cfg, const le_gaussians* g, const le_gaussian_grads* m,
                     const le_gaussian_grads* v, const float* acc, const int32_t* cnt, const int32_t* max_radius,
                     const float* noise,
                     int64_t n_cap, const le_gaussian_grads* g_out, const le_gaussian_grads* m_out,
                     const le_gaussian_grads* v_out, int64_t* n_out, void* workspace, size_t workspace_bytes,
                     void* stream);

/* ---------------------------------------------------------------------------
 * Training helpers (Sec. 4).
 * le_rgb_l1: L = mean |img - target| over n values, loss[0] = L (device
 *   scalar, overwritten), grad = sign(img - target)/n (the 3DGS RGB loss's
 *   L1 term; reading).
 * le_adam: in-place Adam over one flat buffer (lr 1e-3 and betas (0.9,
 *   0.999) in the paper; eps is a reading), step >= 1, then clamp to
 *   [clamp_lo, clamp_hi] (pass -inf/+inf for none; u uses [0,1], Sec. 3.4.2). */
le_status le_rgb_l1(int64_t n, const float* img, const float* target, float* loss, float* grad, void* stream);

/* le_rgb_loss -- the full RGB loss of 3D Gaussian Splatting, which Sec. 4
 * keeps ("the same RGB loss"; reading, the paper does not restate it):
 *   L = (1 - lambda_ssim) L1 + lambda_ssim (1 - SSIM)   (3DGS: lambda_ssim = 0.2)
 * SSIM per channel with an 11 x 11 Gaussian window (sigma 1.5), zero padding
 * outside the image, C1 = 0.01^2, C2 = 0.03^2, mean over pixels and channels.
 *   img, target [3,H,W]; loss [3] out = (L, L1, SSIM); grad [3,H,W] out = dL/dimg;
 *   workspace: le_rgb_loss_workspace(W, H) bytes (the three per-pixel SSIM
 *   partial-derivative maps of every channel).
 * Errors: LE_ERR_INVALID_ARG (null pointers, bad size, lambda outside [0,1]). */
le_status le_rgb_loss_workspace(int32_t W, int32_t H, size_t* bytes);
le_status le_rgb_loss(int32_t W, int32_t H, const float* img, const float* target, float lambda_ssim, float* loss,
                      float* grad, void* workspace, size_t workspace_bytes, void* stream);
le_status le_adam(int64_t n, float* param, const float* grad, float* m, float* v, int32_t step, float lr,
                  float beta1, float beta2, float eps, float clamp_lo, float clamp_hi, void* stream);

/* le_device_status -- synchronizes `stream`, then reports whether any
 * tensor-core kernel (fused decode / query) gave up on a bounded wait since the
 * last call: LE_ERR_TIMEOUT (and clears the record) or LE_OK.  Such a kernel
 * stops issuing work, frees its tensor memory and returns; its outputs are
 * then incomplete. */
le_status le_device_status(void* stream);

/* le_selftest_bounded_wait -- exercises that failure path on purpose: one
 * kernel waits on a barrier that nothing ever completes, gives up after the
 * bounded wait (about a second) and records it, so the next le_device_status
 * returns LE_ERR_TIMEOUT.  The GPU context stays usable. */
le_status le_selftest_bounded_wait(void* stream);

/* Message for the last error on the calling thread (static storage). */
const char* le_last_error(void);
/* Number of kernel launches this library issued on the calling thread since the
 * last le_reset_launch_count(). */
int64_t le_launch_count(void);
void le_reset_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* LEG_H */
