/*
 * Oracle open-vocabulary relevancy (FP64).  Test infrastructure only.
 *
 * supp. Sec. "Inference": M_infer = softmax(D_MLP(R_s)) gives per pixel a
 * distribution p over the N codebook entries; the language feature map is
 * F = M_infer S (S the N x d codebook); objects are found by the relevancy
 * of F against a text prompt "in accordance with LERF".  Reading of that
 * relevancy (LERF's published definition, temperature 1):
 *   phi   = F_clip / |F_clip|        F_clip = the first d_clip (=512) dims of F
 *   rel_j = min_k exp(phi.q_j) / (exp(phi.q_j) + exp(phi.n_k))
 * for unit text embeddings q_j and canonical negatives n_k.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

void orc_query(int P, int ncb, const double* prob, const float* codebook, int d, int d_clip,
               const float* text, int Q, const float* negs, int n_neg, double* rel)
{
#pragma omp parallel
    {
        double* F = (double*)malloc(sizeof(double) * d_clip);
#pragma omp for schedule(static)
        for (int p = 0; p < P; ++p) {
            for (int e = 0; e < d_clip; ++e) F[e] = 0;
            for (int i = 0; i < ncb; ++i) {
                const double w = prob[(size_t)i * P + p];
                for (int e = 0; e < d_clip; ++e) F[e] += w * codebook[(size_t)i * d + e];
            }
            double n2 = 0;
            for (int e = 0; e < d_clip; ++e) n2 += F[e] * F[e];
            const double inv = 1.0 / sqrt(n2);
            for (int j = 0; j < Q; ++j) {
                double sq = 0;
                for (int e = 0; e < d_clip; ++e) sq += F[e] * inv * text[(size_t)j * d_clip + e];
                double best = INFINITY;
                for (int k = 0; k < n_neg; ++k) {
                    double sn = 0;
                    for (int e = 0; e < d_clip; ++e) sn += F[e] * inv * negs[(size_t)k * d_clip + e];
                    const double r = exp(sq) / (exp(sq) + exp(sn));
                    if (r < best) best = r;
                }
                rel[(size_t)j * P + p] = best;
            }
        }
        free(F);
    }
}

/* The language feature map itself, F[p] = sum_i prob[i][p] S_i (supp. Sec.
 * "Inference": F = M_infer S), FP64: F [P][d]. */
void orc_feature_map(int P, int ncb, const double* prob, const float* codebook, int d, double* F)
{
#pragma omp parallel for schedule(static)
    for (int p = 0; p < P; ++p) {
        double* f = F + (size_t)p * d;
        for (int e = 0; e < d; ++e) f[e] = 0.0;
        for (int i = 0; i < ncb; ++i) {
            const double w = prob[(size_t)i * P + p];
            for (int e = 0; e < d; ++e) f[e] += w * codebook[(size_t)i * d + e];
        }
    }
}
