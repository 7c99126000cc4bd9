/*
 * Oracle quantisation of language features (FP64).  Test infrastructure only.
 *
 * Sec. 3.3 "Quantization of Language Features" and the supplementary section
 * "Load Balancing Loss":
 *   D(F, f_j) = cos(F^C, f_j^C) + lambda_D cos(F^D, f_j^D)             Eq. eq:q_dist
 *               (F^C: the CLIP part, dims [0, d_clip); F^D: the DINO part)
 *   m = argmax_j D(F, f_j),  F_hat = f_m                         Eqs. eq:quant, eq:q_dist
 *   L_cos(F_i) = (1 - cos(F_i^C, F_hat_i^C)) + lambda_D (1 - cos(F_i^D, F_hat_i^D))
 *                                                                  Eq. eq:q_loss_cos
 *   r = sum_i onehot(m_i) / K,  p = sum_i softmax(D(F_i, S)) / K
 *   L_lb = sum_j r_j p_j                                           Eq. eq:q_loss_lb
 *   L_q = lambda_cos L_cos + lambda_lb L_lb                         Eq. eq:q_loss_cb
 * Readings: L_cos of a batch is the mean over its K features; argmax ties go
 * to the lowest index; the gradient treats r as a constant (it counts argmax
 * winners and has no derivative) and is taken with respect to the codebook
 * values the distances use.
 *
 * Precision: FP64.  The features arrive as BF16 bit patterns (converted
 * exactly); with round_codebook = 1 the FP32 codebook is first rounded to
 * BF16 (round to nearest, ties to even) -- the operands the tensor-core path
 * multiplies -- otherwise it is used as given (finite-difference checks).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* FP32 -> BF16 bits, round to nearest even (NaN not expected). */
uint16_t orc_bf16_bits(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

void orc_bf16_bits_array(int64_t n, const float* x, uint16_t* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_bf16_bits(x[i]);
}

double orc_bf16_value(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double dot(const double* a, const double* b, int n)
{
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* D [K][N] (nullable), m [K], r [N], p [N], loss [3] = (L_q, L_cos, L_lb);
 * grad_S [N][d] (nullable): dL_q / d(codebook as used). */
void orc_quantize(int K, int N, int d, int d_clip, const uint16_t* F_bf16, const double* S_in, int round_codebook,
                  double lambda_d, double lambda_cos, double lambda_lb, double* D_out, int32_t* m_out, double* r_out,
                  double* p_out, double* loss_out, double* grad_S)
{
    const int dd = d - d_clip;
    double* S = (double*)malloc(sizeof(double) * (size_t)N * d);
    double* nS = (double*)malloc(sizeof(double) * 2 * N);          /* |f_j^C|, |f_j^D| */
    for (size_t e = 0; e < (size_t)N * d; ++e)
        S[e] = round_codebook ? orc_bf16_value(orc_bf16_bits((float)S_in[e])) : S_in[e];
    for (int j = 0; j < N; ++j) {
        nS[2 * j] = sqrt(dot(S + (size_t)j * d, S + (size_t)j * d, d_clip));
        nS[2 * j + 1] = sqrt(dot(S + (size_t)j * d + d_clip, S + (size_t)j * d + d_clip, dd));
    }
    double* D = (double*)malloc(sizeof(double) * (size_t)K * N);
    double* cC = (double*)malloc(sizeof(double) * (size_t)K * N);   /* the two cosines, for the gradient */
    double* cD = (double*)malloc(sizeof(double) * (size_t)K * N);
    double* nF = (double*)malloc(sizeof(double) * 2 * (size_t)K);
    double lcos = 0.0;
#pragma omp parallel
    {
        double* x = (double*)malloc(sizeof(double) * d);
#pragma omp for schedule(static) reduction(+ : lcos)
        for (int i = 0; i < K; ++i) {
            for (int e = 0; e < d; ++e) x[e] = orc_bf16_value(F_bf16[(size_t)i * d + e]);
            const double nc = sqrt(dot(x, x, d_clip)), nd = sqrt(dot(x + d_clip, x + d_clip, dd));
            nF[2 * (size_t)i] = nc;
            nF[2 * (size_t)i + 1] = nd;
            int best = 0;
            for (int j = 0; j < N; ++j) {
                const double* f = S + (size_t)j * d;
                const double c1 = dot(x, f, d_clip) / (nc * nS[2 * j]);
                const double c2 = dot(x + d_clip, f + d_clip, dd) / (nd * nS[2 * j + 1]);
                const size_t o = (size_t)i * N + j;
                cC[o] = c1;
                cD[o] = c2;
                D[o] = c1 + lambda_d * c2;
                if (D[o] > D[(size_t)i * N + best]) best = j;
            }
            m_out[i] = best;
            const size_t ob = (size_t)i * N + best;
            lcos += (1.0 - cC[ob]) + lambda_d * (1.0 - cD[ob]);
        }
        free(x);
    }
    /* utilisation ratio r and mean selection probability p */
    for (int j = 0; j < N; ++j) r_out[j] = p_out[j] = 0.0;
    double* sm = (double*)malloc(sizeof(double) * (size_t)K * N);   /* row softmax of D */
    for (int i = 0; i < K; ++i) {
        r_out[m_out[i]] += 1.0;
        double mx = -INFINITY, z = 0.0;
        for (int j = 0; j < N; ++j) mx = fmax(mx, D[(size_t)i * N + j]);
        for (int j = 0; j < N; ++j) z += exp(D[(size_t)i * N + j] - mx);
        for (int j = 0; j < N; ++j) {
            const double s = exp(D[(size_t)i * N + j] - mx) / z;
            sm[(size_t)i * N + j] = s;
            p_out[j] += s;
        }
    }
    double lb = 0.0;
    for (int j = 0; j < N; ++j) {
        r_out[j] /= K;
        p_out[j] /= K;
        lb += r_out[j] * p_out[j];
    }
    lcos /= K;
    loss_out[0] = lambda_cos * lcos + lambda_lb * lb;
    loss_out[1] = lcos;
    loss_out[2] = lb;
    if (D_out) memcpy(D_out, D, sizeof(double) * (size_t)K * N);

    if (grad_S) {
        /* g_ij = dL_q/dD_ij = -lambda_cos/K [j = m_i] + lambda_lb/K s_ij (r_j - sum_k s_ik r_k);
         * d cos(a, b)/db = (a/|a| - cos b/|b|)/|b| for each part, the DINO part weighted by lambda_D. */
        memset(grad_S, 0, sizeof(double) * (size_t)N * d);
        for (int i = 0; i < K; ++i) {
            double sr = 0.0;
            for (int j = 0; j < N; ++j) sr += sm[(size_t)i * N + j] * r_out[j];
            for (int j = 0; j < N; ++j) {
                const size_t o = (size_t)i * N + j;
                double g = lambda_lb / K * sm[o] * (r_out[j] - sr);
                if (j == m_out[i]) g -= lambda_cos / K;
                if (g == 0.0) continue;
                const double* f = S + (size_t)j * d;
                double* G = grad_S + (size_t)j * d;
                for (int e = 0; e < d_clip; ++e) {
                    const double a = orc_bf16_value(F_bf16[(size_t)i * d + e]) / nF[2 * (size_t)i];
                    G[e] += g * (a - cC[o] * f[e] / nS[2 * j]) / nS[2 * j];
                }
                for (int e = d_clip; e < d; ++e) {
                    const double a = orc_bf16_value(F_bf16[(size_t)i * d + e]) / nF[2 * (size_t)i + 1];
                    G[e] += g * lambda_d * (a - cD[o] * f[e] / nS[2 * j + 1]) / nS[2 * j + 1];
                }
            }
        }
    }
    free(sm);
    free(nF);
    free(cD);
    free(cC);
    free(D);
    free(nS);
    free(S);
}
