/*
 * FP64 CPU oracle for the Language Embedded 3D Gaussians hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code; only the tests, `__graft_entry__.smoke()` and the
 * benchmark's CPU-baseline leg do.  It shares no header, helper or constant
 * table with the CUDA library: it is a plain, slow, single-pass restatement of
 * what the method computes, written from the paper's definitions.
 *
 * What it follows:
 *   - rendering I = R(p, Sigma, c, alpha; p_cam)                 Eq. 1 (eq:render), Sec. 3.1
 *     (projection, tiling and compositing are the 3D Gaussian Splatting
 *      rasterizer that Sec. 4 says was reused; its constants are readings)
 *   - semantic feature / uncertainty rendering R_s, R_u             Sec. 3.4.1, 3.4.2
 *   - decoder D_MLP (1x1 convs 8 -> h1 -> h2 -> N)     Eq. 8 (eq:lem_dec), supp. Tab. dmlp
 *   - L_CE with uncertainty weighting, L_u, L_s    Eqs. 10-12 (eq:lem_loss_ce1, _uncer, eq:lem_loss)
 *   - inference M_infer = softmax(D_MLP(R_s)), F = M_infer S, relevancy   supp. Sec. "Inference"
 *   - Adam with lr 1e-3, betas (0.9, 0.999)                          Sec. 4
 *   - RGB loss (1 - lambda) L1 + lambda D-SSIM (3DGS's, kept by Sec. 4)
 *   - adaptive density control: clone / split / prune (3DGS's, kept by Sec. 4)
 *   - adaptive spatial smoothing: MLP(PE(p)), L_smo       Sec. 3.4 (eq:lem_fmlp, eq:lem_loss_mlp)
 *   - quantisation of language features: mixed cosine argmax, L_cos,
 *     load balancing L_lb, L_q           Sec. 3.3 (eq:q_dist .. eq:q_loss_cb), supp. Sec. 1
 *
 * Precision: FP64 everywhere except the "key path" (keypath.c), which decides
 * integers (culling, tile rectangle, sort key) and therefore is evaluated in
 * FP32 with a fixed sequence of IEEE operations that the GPU side also
 * follows (see keypath.c).
 *
 * Layouts: per-Gaussian arrays are structure-of-arrays, images are planar
 * [channel][row][col].  Pixel (i, j) is sampled at integer coordinates.
 */
#ifndef LEG_ORACLE_H
#define LEG_ORACLE_H
#include <stdint.h>

#define ORC_TILE 16
#define ORC_DFEAT 8
#define ORC_NCH 12          /* rgb 3 + semantic feature 8 + uncertainty 1 */

typedef struct {
    float view[12];         /* world->camera [R|t], row-major */
    float campos[3];        /* camera centre in world coordinates */
    float fx, fy, cx, cy;
    int32_t W, H;
    float near_z;
    float bg[3];
} orc_cam;

/* keypath.c */
float orc_exp_f32(float x);
float orc_ln_up_f32(float x);
void orc_keypath(int N, const float* means, const float* log_scales, const float* quats,
                 const float* opacity_raw, const orc_cam* cam, float* depth, float* mean2d, float* cov2d,
                 int32_t* radius, int32_t* rect, int32_t* tiles, float* ell /* [N][8] */);

/* sh.c */
int orc_sh_count(int deg);
void orc_sh_basis(int deg, const double dir[3], double* Y, double* dY /* nullable, [n][3] */);

/* project.c */
void orc_project(int N, int deg, const double* means, const double* log_scales, const double* quats,
                 const double* opacity_raw, const double* sh, const orc_cam* cam, const int32_t* tiles,
                 double* mean2d, double* depth, double* cov2d, double* conic, double* opacity,
                 double* rgb, uint8_t* clamp);
void orc_project_bwd(int N, int deg, const double* means, const double* log_scales, const double* quats,
                     const double* opacity_raw, const double* sh, const orc_cam* cam, const int32_t* tiles,
                     const double* d_mean2d, const double* d_conic, const double* d_opacity,
                     const double* d_rgb, double* d_means, double* d_log_scales, double* d_quats,
                     double* d_opacity_raw, double* d_sh);

/* binning.c */
void orc_row_span(const float* E, const int32_t* r, int ty, int* xl, int* xr);
int64_t orc_bin(int N, const orc_cam* cam, const float* depth, const int32_t* rect, const int32_t* tiles,
                const float* ell /* nullable: whole rectangles */, uint64_t* keys, uint32_t* vals,
                uint32_t* ranges);
int64_t orc_bin_count(int N, const int32_t* rect, const int32_t* tiles, const float* ell /* nullable */);
int orc_tile_list(int N, const float* depth, const int32_t* rect, const int32_t* tiles,
                  const float* ell /* nullable */, int tx, int ty, uint32_t* out);

/* composite.c */
void orc_render(const orc_cam* cam, int N, const uint32_t* vals, const uint32_t* ranges,
                const double* mean2d, const double* conic, const double* opacity, const double* rgb,
                const float* feat, const float* unc, int x0, int y0, int x1, int y1,
                double* out_rgb, double* out_feat, double* out_unc, double* T_final,
                int32_t* n_contrib, uint8_t* flip);
void orc_render_bwd(const orc_cam* cam, int N, const uint32_t* vals, const uint32_t* ranges,
                    const double* mean2d, const double* conic, const double* opacity, const double* rgb,
                    const float* feat, const float* unc, int x0, int y0, int x1, int y1,
                    const double* dL_drgb, const double* dL_dfeat, const double* dL_dunc,
                    double* d_mean2d, double* d_conic, double* d_opacity, double* d_rgb,
                    double* d_feat, double* d_unc);

/* decoder.c */
void orc_decoder_fwd(int P, int d_in, int h1, int h2, int ncb, const double* feat,
                     const double* W1, const double* b1, const double* W2, const double* b2,
                     const double* W3, const double* b3, double* logits);
void orc_softmax_argmax(int P, int ncb, const double* logits, double* prob, int32_t* argmax);
void orc_decoder_loss(int P, int d_in, int h1, int h2, int ncb, const double* feat, const double* unc,
                      const int32_t* target, const double* W1, const double* b1, const double* W2,
                      const double* b2, const double* W3, const double* b3, double lambda_ce,
                      double lambda_u, double* loss, double* d_feat, double* d_unc, double* dW1,
                      double* db1, double* dW2, double* db2, double* dW3, double* db3);

/* query.c */
void orc_query(int P, int ncb, const double* prob, const float* codebook, int d, int d_clip,
               const float* text, int Q, const float* negs, int n_neg, double* rel);

/* train.c */
double orc_l1(int64_t n, const double* img, const float* target, double* grad);
void orc_adam(int64_t n, double* param, const double* grad, double* m, double* v, int step,
              double lr, double b1, double b2, double eps);

/* query.c: the feature map */
void orc_feature_map(int P, int ncb, const double* prob, const float* codebook, int d, double* F);

/* ssim.c */
void orc_rgb_loss(int W, int H, const double* img, const double* target, double lambda, double* loss, double* grad,
                  double* smap);

/* densify.c */
int64_t orc_densify_plan(int n, const float* log_scales, const float* opacity_raw, const float* acc,
                         const int32_t* cnt, const int32_t* max_radius, float grad_thresh, float log_big,
                         float logit_min, float max_screen, float log_world, int32_t* kind);
void orc_densify_stats(int n, const float* grad_mean2d, const int32_t* radius, float* acc, int32_t* cnt,
                       int32_t* max_radius);
void orc_opacity_reset(int n, float* opacity_raw, float* m, float* v, float logit_max);
void orc_split_mean(const float* mu, const float* log_s, const float* q, const float* nz, double* out);

/* quant.c */
uint16_t orc_bf16_bits(float x);
void orc_bf16_bits_array(int64_t n, const float* x, uint16_t* out);
double orc_bf16_value(uint16_t b);
void orc_quantize(int K, int N, int d, int d_clip, const uint16_t* F_bf16, const double* S_in, int round_codebook,
                  double lambda_d, double lambda_cos, double lambda_lb, double* D_out, int32_t* m_out, double* r_out,
                  double* p_out, double* loss_out, double* grad_S);

/* smooth.c */
void orc_smooth(int n, const double* means, const double* feat, const double* unc, const double* W1,
                const double* b1, const double* W2, const double* b2, const double* W3, const double* b3,
                const double* W4, const double* b4, double w_s, double lambda, double* s_mlp, double* loss,
                double* d_feat, double* dW1, double* db1, double* dW2, double* db2, double* dW3, double* db3,
                double* dW4, double* db4);

#endif
