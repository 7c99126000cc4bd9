/*
 * Oracle semantic decoder, softmax, cross-entropy and its adjoint (FP64).
 * Test infrastructure only; see oracle.h.
 *
 * D_MLP (Eq. 8, eq:lem_dec; supp. Tab. dmlp): three 1x1 convolutions, i.e. a
 * per-pixel MLP  z = W3 relu(W2 relu(W1 f + b1) + b2) + b3,  f in R^8 the
 * rendered semantic feature R_s, z in R^N the logits over the codebook.
 * Weights are [out][in] row-major.  Maps are planar: feat [d_in][P],
 * logits / prob [N][P].
 *
 * Loss (Eqs. 9-12):
 *   CE_px = logsumexp(z) - z[M_px]
 *   L_CE  = sum_px CE_px (1 - R_u,px) / P,  L_u = sum_px R_u,px / P
 *   L_s   = lambda_CE L_CE + lambda_u L_u
 * The uncertainty weighting is differentiated too (Sec. 3.4.2: inconsistent
 * indices are meant to raise u):
 *   dL/dz    = lambda_CE (1 - u)/P (softmax(z) - onehot(M))
 *   dL/du_px = (lambda_u - lambda_CE CE_px) / P
 * ReLU derivative: 1 where the pre-activation is > 0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static void mlp_pixel(int d_in, int h1, int h2, int ncb, const double* f, const double* W1, const double* b1,
                      const double* W2, const double* b2, const double* W3, const double* b3, double* a1,
                      double* a2, double* z)
{
    for (int o = 0; o < h1; ++o) {
        double v = b1[o];
        for (int i = 0; i < d_in; ++i) v += W1[o * d_in + i] * f[i];
        a1[o] = v > 0 ? v : 0;
    }
    for (int o = 0; o < h2; ++o) {
        double v = b2[o];
        for (int i = 0; i < h1; ++i) v += W2[o * h1 + i] * a1[i];
        a2[o] = v > 0 ? v : 0;
    }
    for (int o = 0; o < ncb; ++o) {
        double v = b3[o];
        for (int i = 0; i < h2; ++i) v += W3[o * h2 + i] * a2[i];
        z[o] = v;
    }
}

void orc_decoder_fwd(int P, int d_in, int h1, int h2, int ncb, const double* feat,
                     const double* W1, const double* b1, const double* W2, const double* b2,
                     const double* W3, const double* b3, double* logits)
{
#pragma omp parallel
    {
        double* buf = (double*)malloc(sizeof(double) * (d_in + h1 + h2 + ncb));
        double *f = buf, *a1 = f + d_in, *a2 = a1 + h1, *z = a2 + h2;
#pragma omp for schedule(static)
        for (int p = 0; p < P; ++p) {
            for (int i = 0; i < d_in; ++i) f[i] = feat[(size_t)i * P + p];
            mlp_pixel(d_in, h1, h2, ncb, f, W1, b1, W2, b2, W3, b3, a1, a2, z);
            for (int o = 0; o < ncb; ++o) logits[(size_t)o * P + p] = z[o];
        }
        free(buf);
    }
}

void orc_softmax_argmax(int P, int ncb, const double* logits, double* prob, int32_t* argmax)
{
    for (int p = 0; p < P; ++p) {
        double m = logits[p];
        int am = 0;
        for (int o = 1; o < ncb; ++o)
            if (logits[(size_t)o * P + p] > m) {
                m = logits[(size_t)o * P + p];
                am = o;
            }
        double s = 0;
        for (int o = 0; o < ncb; ++o) s += exp(logits[(size_t)o * P + p] - m);
        if (prob)
            for (int o = 0; o < ncb; ++o) prob[(size_t)o * P + p] = exp(logits[(size_t)o * P + p] - m) / s;
        if (argmax) argmax[p] = am;
    }
}

void orc_decoder_loss(int P, int d_in, int h1, int h2, int ncb, const double* feat, const double* unc,
                      const int32_t* target, const double* W1, const double* b1, const double* W2,
                      const double* b2, const double* W3, const double* b3, double lambda_ce,
                      double lambda_u, double* loss, double* d_feat, double* d_unc, double* dW1,
                      double* db1, double* dW2, double* db2, double* dW3, double* db3)
{
    memset(dW1, 0, sizeof(double) * h1 * d_in);
    memset(db1, 0, sizeof(double) * h1);
    memset(dW2, 0, sizeof(double) * h2 * h1);
    memset(db2, 0, sizeof(double) * h2);
    memset(dW3, 0, sizeof(double) * ncb * h2);
    memset(db3, 0, sizeof(double) * ncb);
    double* buf = (double*)malloc(sizeof(double) * (d_in + 2 * h1 + 2 * h2 + 2 * ncb));
    double *f = buf, *a1 = f + d_in, *a2 = a1 + h1, *z = a2 + h2, *dz = z + ncb, *g2 = dz + ncb, *g1 = g2 + h2;
    double Lce = 0, Lu = 0;
    for (int p = 0; p < P; ++p) {
        for (int i = 0; i < d_in; ++i) f[i] = feat[(size_t)i * P + p];
        mlp_pixel(d_in, h1, h2, ncb, f, W1, b1, W2, b2, W3, b3, a1, a2, z);
        double m = z[0];
        for (int o = 1; o < ncb; ++o) m = z[o] > m ? z[o] : m;
        double s = 0;
        for (int o = 0; o < ncb; ++o) s += exp(z[o] - m);
        const double lse = m + log(s);
        const double ce = lse - z[target[p]];
        const double u = unc[p];
        Lce += ce * (1 - u);
        Lu += u;
        d_unc[p] = (lambda_u - lambda_ce * ce) / P;
        const double w = lambda_ce * (1 - u) / P;
        for (int o = 0; o < ncb; ++o) dz[o] = w * (exp(z[o] - lse) - (o == target[p] ? 1.0 : 0.0));
        /* layer 3 */
        for (int o = 0; o < ncb; ++o) {
            db3[o] += dz[o];
            for (int i = 0; i < h2; ++i) dW3[o * h2 + i] += dz[o] * a2[i];
        }
        for (int i = 0; i < h2; ++i) {
            double v = 0;
            for (int o = 0; o < ncb; ++o) v += W3[o * h2 + i] * dz[o];
            g2[i] = a2[i] > 0 ? v : 0;
        }
        /* layer 2 */
        for (int o = 0; o < h2; ++o) {
            db2[o] += g2[o];
            for (int i = 0; i < h1; ++i) dW2[o * h1 + i] += g2[o] * a1[i];
        }
        for (int i = 0; i < h1; ++i) {
            double v = 0;
            for (int o = 0; o < h2; ++o) v += W2[o * h1 + i] * g2[o];
            g1[i] = a1[i] > 0 ? v : 0;
        }
        /* layer 1 */
        for (int o = 0; o < h1; ++o) {
            db1[o] += g1[o];
            for (int i = 0; i < d_in; ++i) dW1[o * d_in + i] += g1[o] * f[i];
        }
        for (int i = 0; i < d_in; ++i) {
            double v = 0;
            for (int o = 0; o < h1; ++o) v += W1[o * d_in + i] * g1[o];
            d_feat[(size_t)i * P + p] = v;
        }
    }
    loss[0] = Lce / P;
    loss[1] = Lu / P;
    free(buf);
}
