/*
 * CPU oracle of the cost-model network -- TEST INFRASTRUCTURE ONLY (used by
 * the test suite to check the CUDA forward/backward/Adam kernels).
 *
 * FP64 forward pass, mean-squared-error loss and its exact gradient by
 * reverse-mode differentiation of
 *     y = w4 . g(W3 g(W2 g(W1 x + b1) + b2) + b3) + b4,
 *     g(z) = z (1 + erf(z / sqrt 2)) / 2,   loss = mean (y - t)^2,
 * with the parameter layout W1[64][D], b1[64], W2[64][64], b2[64],
 * W3[64][64], b3[64], w4[64], b4 (floats in, doubles inside), and one
 * Adam step (Kingma and Ba, 2015, with bias correction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HID 64

static double gel(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }
static const double kPi = 3.14159265358979323846;
static double geld(double z) { return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * kPi); }

int64_t oracle_mlp_param_count(int D) { return (int64_t)HID * D + HID + 2 * ((int64_t)HID * HID + HID) + HID + 1; }

/* Returns the loss; writes predictions to y (may be NULL) and the gradient
 * of the loss to grad (may be NULL), both as doubles. */
double oracle_mlp_loss_grad(const float *P, int D, const float *X, const float *T, int64_t n, double *y,
                            double *grad)
{
    const int64_t np = oracle_mlp_param_count(D);
    double *p = (double *)malloc(sizeof(double) * np);
    for (int64_t i = 0; i < np; i++) p[i] = P[i];
    const double *W1 = p, *b1 = W1 + HID * D, *W2 = b1 + HID, *b2 = W2 + HID * HID, *W3 = b2 + HID;
    const double *b3 = W3 + HID * HID, *w4 = b3 + HID, *b4 = w4 + HID;
    if (grad) memset(grad, 0, sizeof(double) * np);
    double *gW1 = grad, *gb1 = grad ? gW1 + HID * D : NULL, *gW2 = grad ? gb1 + HID : NULL;
    double *gb2 = grad ? gW2 + HID * HID : NULL, *gW3 = grad ? gb2 + HID : NULL;
    double *gb3 = grad ? gW3 + HID * HID : NULL, *gw4 = grad ? gb3 + HID : NULL, *gb4 = grad ? gw4 + HID : NULL;
    double loss = 0.0;
    for (int64_t s = 0; s < n; s++) {
        const float *x = X + s * D;
        double z1[HID], a1[HID], z2[HID], a2[HID], z3[HID], a3[HID];
        for (int j = 0; j < HID; j++) {
            double acc = b1[j];
            for (int k = 0; k < D; k++) acc += W1[j * D + k] * x[k];
            z1[j] = acc;
            a1[j] = gel(acc);
        }
        for (int j = 0; j < HID; j++) {
            double acc = b2[j];
            for (int k = 0; k < HID; k++) acc += W2[j * HID + k] * a1[k];
            z2[j] = acc;
            a2[j] = gel(acc);
        }
        for (int j = 0; j < HID; j++) {
            double acc = b3[j];
            for (int k = 0; k < HID; k++) acc += W3[j * HID + k] * a2[k];
            z3[j] = acc;
            a3[j] = gel(acc);
        }
        double out = b4[0];
        for (int j = 0; j < HID; j++) out += w4[j] * a3[j];
        if (y) y[s] = out;
        const double e = out - T[s];
        loss += e * e / (double)n;
        if (!grad) continue;
        const double dy = 2.0 * e / (double)n;
        double d3[HID], d2[HID], d1[HID];
        gb4[0] += dy;
        for (int j = 0; j < HID; j++) {
            gw4[j] += dy * a3[j];
            d3[j] = dy * w4[j] * geld(z3[j]);
        }
        for (int j = 0; j < HID; j++) {
            gb3[j] += d3[j];
            for (int k = 0; k < HID; k++) gW3[j * HID + k] += d3[j] * a2[k];
        }
        for (int k = 0; k < HID; k++) {
            double acc = 0.0;
            for (int j = 0; j < HID; j++) acc += W3[j * HID + k] * d3[j];
            d2[k] = acc * geld(z2[k]);
        }
        for (int j = 0; j < HID; j++) {
            gb2[j] += d2[j];
            for (int k = 0; k < HID; k++) gW2[j * HID + k] += d2[j] * a1[k];
        }
        for (int k = 0; k < HID; k++) {
            double acc = 0.0;
            for (int j = 0; j < HID; j++) acc += W2[j * HID + k] * d2[j];
            d1[k] = acc * geld(z1[k]);
        }
        for (int j = 0; j < HID; j++) {
            gb1[j] += d1[j];
            for (int k = 0; k < D; k++) gW1[j * D + k] += d1[j] * x[k];
        }
    }
    free(p);
    return loss;
}

/* One Adam step in FP64 on double arrays (in place). */
void oracle_adam(double *p, const double *g, double *m, double *v, int64_t np, double lr, double b1, double b2,
                 double eps, int step)
{
    const double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
    for (int64_t i = 0; i < np; i++) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
