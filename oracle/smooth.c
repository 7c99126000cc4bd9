/*
 * Oracle adaptive spatial smoothing (FP64).  Test infrastructure only.
 *
 * Sec. 3.4 "Adaptive spatial smoothing loss", Eqs. eq:lem_fmlp and
 * eq:lem_loss_mlp, supplementary Tab. pemlp:
 *   s_MLP = MLP(PE(p)),  PE of frequency 0 (output size 3: the position itself),
 *   MLP: 3 -> 128 (ReLU) -> 128 (ReLU) -> 128 (ReLU) -> 8 (linear), weights [out][in]
 *   L_smo = |s_MLP - s_G*|_2 + max(u_G*, w_s) |s_MLP* - s_G|_2      (* = stop gradient)
 * Readings: the loss of a set of n Gaussians is the mean of the per-Gaussian
 * terms, times lambda_smo (Eq. eq:loss); |.|_2 is the plain (not squared) norm,
 * whose gradient at a zero difference is taken as 0; no gradient reaches the
 * positions or u.  So per Gaussian, with n_i = |s_MLP - s_G|:
 *   L_i = (1 + max(u_i, w_s)) n_i
 *   dL/ds_MLP = lambda/n (s_MLP - s_G)/n_i                    (first term only)
 *   dL/ds_G   = -lambda/n max(u_i, w_s) (s_MLP - s_G)/n_i      (second term only)
 * and dL/ds_MLP is back-propagated through the MLP to every weight and bias.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

#define H 128
#define DS 8

/* d_feat [n][8] out; dW1 [128][3], db1 [128], dW2 [128][128], db2, dW3, db3,
 * dW4 [8][128], db4 [8] out; s_mlp [n][8] out (nullable); loss [1] out. */
void orc_smooth(int n, const double* means, const double* feat, const double* unc, const double* W1,
                const double* b1, const double* W2, const double* b2, const double* W3, const double* b3,
                const double* W4, const double* b4, double w_s, double lambda, double* s_mlp, double* loss,
                double* d_feat, double* dW1, double* db1, double* dW2, double* db2, double* dW3, double* db3,
                double* dW4, double* db4)
{
    memset(dW1, 0, sizeof(double) * H * 3);
    memset(db1, 0, sizeof(double) * H);
    memset(dW2, 0, sizeof(double) * H * H);
    memset(db2, 0, sizeof(double) * H);
    memset(dW3, 0, sizeof(double) * H * H);
    memset(db3, 0, sizeof(double) * H);
    memset(dW4, 0, sizeof(double) * DS * H);
    memset(db4, 0, sizeof(double) * DS);
    double L = 0.0;
    for (int i = 0; i < n; ++i) {
        const double* x = means + 3 * (size_t)i;
        double h1[H], h2[H], h3[H], z[DS];
        for (int a = 0; a < H; ++a) {
            double s = b1[a];
            for (int k = 0; k < 3; ++k) s += W1[a * 3 + k] * x[k];
            h1[a] = s > 0.0 ? s : 0.0;
        }
        for (int a = 0; a < H; ++a) {
            double s = b2[a];
            for (int k = 0; k < H; ++k) s += W2[a * H + k] * h1[k];
            h2[a] = s > 0.0 ? s : 0.0;
        }
        for (int a = 0; a < H; ++a) {
            double s = b3[a];
            for (int k = 0; k < H; ++k) s += W3[a * H + k] * h2[k];
            h3[a] = s > 0.0 ? s : 0.0;
        }
        for (int c = 0; c < DS; ++c) {
            double s = b4[c];
            for (int k = 0; k < H; ++k) s += W4[c * H + k] * h3[k];
            z[c] = s;
        }
        if (s_mlp)
            for (int c = 0; c < DS; ++c) s_mlp[(size_t)i * DS + c] = z[c];
        double diff[DS], nn = 0.0;
        for (int c = 0; c < DS; ++c) {
            diff[c] = z[c] - feat[(size_t)i * DS + c];
            nn += diff[c] * diff[c];
        }
        nn = sqrt(nn);
        const double wgt = unc[i] > w_s ? unc[i] : w_s;
        L += (1.0 + wgt) * nn;
        double dz[DS];
        for (int c = 0; c < DS; ++c) {
            const double g = nn > 0.0 ? diff[c] / nn * lambda / n : 0.0;
            dz[c] = g;
            d_feat[(size_t)i * DS + c] = -wgt * g;
        }
        /* back through the MLP */
        double d3[H], d2[H], d1[H];
        for (int k = 0; k < H; ++k) {
            double s = 0.0;
            for (int c = 0; c < DS; ++c) s += dz[c] * W4[c * H + k];
            d3[k] = h3[k] > 0.0 ? s : 0.0;
        }
        for (int c = 0; c < DS; ++c) {
            db4[c] += dz[c];
            for (int k = 0; k < H; ++k) dW4[c * H + k] += dz[c] * h3[k];
        }
        for (int k = 0; k < H; ++k) {
            double s = 0.0;
            for (int a = 0; a < H; ++a) s += d3[a] * W3[a * H + k];
            d2[k] = h2[k] > 0.0 ? s : 0.0;
        }
        for (int a = 0; a < H; ++a) {
            db3[a] += d3[a];
            for (int k = 0; k < H; ++k) dW3[a * H + k] += d3[a] * h2[k];
        }
        for (int k = 0; k < H; ++k) {
            double s = 0.0;
            for (int a = 0; a < H; ++a) s += d2[a] * W2[a * H + k];
            d1[k] = h1[k] > 0.0 ? s : 0.0;
        }
        for (int a = 0; a < H; ++a) {
            db2[a] += d2[a];
            for (int k = 0; k < H; ++k) dW2[a * H + k] += d2[a] * h1[k];
        }
        for (int a = 0; a < H; ++a) {
            db1[a] += d1[a];
            for (int k = 0; k < 3; ++k) dW1[a * 3 + k] += d1[a] * x[k];
        }
    }
    loss[0] = lambda * L / n;
}
