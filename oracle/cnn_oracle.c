/*
 * cnn_oracle.c -- plain FP64 CPU statement of the candidate classifier of the
 * DSA-110 NSFRB paper (arXiv 2510.18136, Sec. 2.3: successive convolutional
 * blocks with batch normalisation, a non-linearity and max-pooling, then a
 * small fully connected head with dropout, one logit per candidate, binary
 * cross-entropy, Adam).
 *
 * TEST INFRASTRUCTURE ONLY: the parity oracle for the CUDA classifier
 * kernels; shares no code with them.
 *
 * Network (channels-last, input [B][D][H][W][C0], D = time, H, W = image,
 * C0 = subbands):
 *   4 x { conv3d 3x3x3, zero padding 1, no bias -> batch norm (training: batch
 *         statistics, biased variance, eps 1e-5) -> ReLU -> max-pool 2x2x2 }
 *   flatten (d, h, w, c) -> FC1 (F units, bias) -> ReLU -> dropout(p) ->
 *   FC2 (1 unit, bias) -> logit;  loss = mean BCE-with-logits.
 *
 * Parameter vector (one flat array, in this order):
 *   for l = 0..3: W_l[C_l][27][C_{l-1}] (tap k = (kz*3+ky)*3+kx), gamma_l[C_l], beta_l[C_l]
 *   fc1_w[F][Fin], fc1_b[F], fc2_w[F], fc2_b[1]       (Fin = D/16*H/16*W/16*C_4)
 *
 * Dropout mask: keep unit (b, f) of training step s iff the first word of
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) with counter
 * (b*F + f, s, 0, 0) and key (seed_lo, seed_hi), shifted right by 8 and
 * scaled by 2^-24, is >= p; kept units are scaled by 1/(1-p).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int B, D, H, W, C0;
    int C[4];
    int F;
} orc_cnn_dims;

/* ----------------------------------------------------------- Philox4x32-10 */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Philox4x32 with 10 rounds: the multipliers 0xD2511F53 / 0xCD9E8D57 and the
 * Weyl key increments 0x9E3779B9 / 0xBB67AE85 are those of the published
 * generator. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* keep[b*F + f] = 1/0 for training step `step` */
void orc_dropout_mask(int B, int F, double p, uint32_t step, uint64_t seed, uint8_t *keep)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int b = 0; b < B; ++b)
        for (int f = 0; f < F; ++f) {
            uint32_t ctr[4] = {(uint32_t)(b * F + f), step, 0u, 0u}, out[4];
            orc_philox4x32_10(ctr, key, out);
            double u = (double)(out[0] >> 8) * (1.0 / 16777216.0);
            keep[b * F + f] = (u >= p) ? 1 : 0;
        }
}

/* ----------------------------------------------------------- helpers */

static int64_t n_params_of(const orc_cnn_dims *d)
{
    int64_t n = 0;
    int cin = d->C0;
    for (int l = 0; l < 4; ++l) {
        n += (int64_t)d->C[l] * 27 * cin + 2 * d->C[l];
        cin = d->C[l];
    }
    int fin = (d->D / 16) * (d->H / 16) * (d->W / 16) * d->C[3];
    n += (int64_t)d->F * fin + d->F + d->F + 1;
    return n;
}

int64_t orc_cnn_n_params(const orc_cnn_dims *d) { return n_params_of(d); }

/* y[b][z][y][x][co] = sum_{kz,ky,kx,ci} W[co][k][ci] * in[b][z+kz-1][y+ky-1][x+kx-1][ci] */
static void conv3d(int B, int D, int H, int W, int cin, int cout, const double *in, const double *w,
                   double *out)
{
    for (int b = 0; b < B; ++b)
        for (int z = 0; z < D; ++z)
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x)
                    for (int co = 0; co < cout; ++co) {
                        double acc = 0.0;
                        for (int kz = 0; kz < 3; ++kz)
                            for (int ky = 0; ky < 3; ++ky)
                                for (int kx = 0; kx < 3; ++kx) {
                                    int zz = z + kz - 1, yy = y + ky - 1, xx = x + kx - 1;
                                    if (zz < 0 || zz >= D || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                                    const double *ip = in + ((((int64_t)b * D + zz) * H + yy) * W + xx) * cin;
                                    const double *wp = w + ((int64_t)co * 27 + (kz * 3 + ky) * 3 + kx) * cin;
                                    for (int ci = 0; ci < cin; ++ci) acc += wp[ci] * ip[ci];
                                }
                        out[((((int64_t)b * D + z) * H + y) * W + x) * cout + co] = acc;
                    }
}

/* ----------------------------------------------------------- forward / backward */

/* Round to bfloat16 (nearest, ties to even) and back: the storage format in
 * which the GPU kernels keep pooled activations and back-propagated conv
 * gradients.  With bf16_storage set, the oracle rounds at exactly those
 * places, so that max-pool arg-max decisions are taken on the same values. */
static double round_bf16(double v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

/*
 * Forward and (if grads != NULL) backward of the mean BCE loss.
 *   x[B][D][H][W][C0], labels[B] in {0, 1} (1 = artefact / RFI),
 *   keep[B][F] dropout mask (NULL: no dropout), p its rate.
 *   train != 0: batch statistics; train == 0: running statistics run_mean /
 *   run_var ([sum C_l] each, layer after layer) are used instead (and no
 *   gradient is computed).  When train != 0 and run_mean / run_var are given,
 *   the batch mean and the unbiased batch variance are returned in them.
 * logits[B] receive the outputs; returns the loss (0 if labels == NULL).
 */
/* As below; gmag (optional, with grads) receives for every gradient entry the sum of the
 * magnitudes of the terms that make it up (|terms| of its final sum over samples, voxels or
 * windows), the scale of the rounding error of any computation of that sum. */
double orc_cnn_forward_backward_mag(const orc_cnn_dims *d, const double *params, const double *x,
                                    const double *labels, const uint8_t *keep, double p, int train,
                                    double *run_mean, double *run_var, double *logits, double *grads,
                                    int bf16_storage, double *gmag)
{
    const int B = d->B;
    int dims[5][4];   /* per stage: D, H, W, C of the activation entering conv l (stage 4 = pooled output) */
    dims[0][0] = d->D; dims[0][1] = d->H; dims[0][2] = d->W; dims[0][3] = d->C0;
    for (int l = 0; l < 4; ++l) {
        dims[l + 1][0] = dims[l][0] / 2; dims[l + 1][1] = dims[l][1] / 2; dims[l + 1][2] = dims[l][2] / 2;
        dims[l + 1][3] = d->C[l];
    }
    const double eps = 1e-5;
    /* parameter offsets */
    int64_t off_w[4], off_g[4], off_b[4], o = 0;
    for (int l = 0; l < 4; ++l) {
        off_w[l] = o; o += (int64_t)d->C[l] * 27 * dims[l][3];
        off_g[l] = o; o += d->C[l];
        off_b[l] = o; o += d->C[l];
    }
    const int fin = dims[4][0] * dims[4][1] * dims[4][2] * dims[4][3];
    const int F = d->F;
    int64_t off_f1w = o; o += (int64_t)F * fin;
    int64_t off_f1b = o; o += F;
    int64_t off_f2w = o; o += F;
    int64_t off_f2b = o; o += 1;

    /* activations */
    double *act[5], *yconv[4], *yhat[4], *zpre[4], *mean[4], *rstd[4];
    int64_t nact[5], npos[4];
    for (int s = 0; s < 5; ++s) {
        nact[s] = (int64_t)B * dims[s][0] * dims[s][1] * dims[s][2] * dims[s][3];
        act[s] = (double *)malloc(sizeof(double) * (size_t)nact[s]);
    }
    memcpy(act[0], x, sizeof(double) * (size_t)nact[0]);
    int64_t rs_off = 0;
    for (int l = 0; l < 4; ++l) {
        const int D = dims[l][0], H = dims[l][1], W = dims[l][2], cin = dims[l][3], cout = d->C[l];
        npos[l] = (int64_t)B * D * H * W;
        const int64_t n = npos[l] * cout;
        yconv[l] = (double *)malloc(sizeof(double) * (size_t)n);
        yhat[l] = (double *)malloc(sizeof(double) * (size_t)n);
        zpre[l] = (double *)malloc(sizeof(double) * (size_t)n);
        mean[l] = (double *)calloc((size_t)cout, sizeof(double));
        rstd[l] = (double *)calloc((size_t)cout, sizeof(double));
        conv3d(B, D, H, W, cin, cout, act[l], params + off_w[l], yconv[l]);
        for (int c = 0; c < cout; ++c) {
            double mu, var;
            if (train) {
                double s = 0.0;
                for (int64_t q = 0; q < npos[l]; ++q) s += yconv[l][q * cout + c];
                mu = s / (double)npos[l];
                double v = 0.0;
                for (int64_t q = 0; q < npos[l]; ++q) {
                    double t = yconv[l][q * cout + c] - mu;
                    v += t * t;
                }
                var = v / (double)npos[l];
                if (run_mean) run_mean[rs_off + c] = mu;
                if (run_var) run_var[rs_off + c] = (npos[l] > 1) ? v / (double)(npos[l] - 1) : 0.0;
            } else {
                mu = run_mean[rs_off + c];
                var = run_var[rs_off + c];
            }
            mean[l][c] = mu;
            rstd[l][c] = 1.0 / sqrt(var + eps);
        }
        const double *g = params + off_g[l], *be = params + off_b[l];
        for (int64_t q = 0; q < npos[l]; ++q)
            for (int c = 0; c < cout; ++c) {
                double h = (yconv[l][q * cout + c] - mean[l][c]) * rstd[l][c];
                yhat[l][q * cout + c] = h;
                zpre[l][q * cout + c] = g[c] * h + be[c];
            }
        /* ReLU + max-pool 2x2x2 (ties: first in (dz, dy, dx) order) */
        const int D2 = dims[l + 1][0], H2 = dims[l + 1][1], W2 = dims[l + 1][2];
        for (int b = 0; b < B; ++b)
            for (int z = 0; z < D2; ++z)
                for (int y = 0; y < H2; ++y)
                    for (int xw = 0; xw < W2; ++xw)
                        for (int c = 0; c < cout; ++c) {
                            double m = -INFINITY;
                            for (int dz = 0; dz < 2; ++dz)
                                for (int dy = 0; dy < 2; ++dy)
                                    for (int dx = 0; dx < 2; ++dx) {
                                        int64_t q = (((int64_t)b * D + 2 * z + dz) * H + 2 * y + dy) * W + 2 * xw + dx;
                                        double v = zpre[l][q * cout + c];
                                        if (v < 0.0) v = 0.0;
                                        if (v > m) m = v;
                                    }
                            act[l + 1][((((int64_t)b * D2 + z) * H2 + y) * W2 + xw) * cout + c] =
                                bf16_storage ? round_bf16(m) : m;
                        }
        rs_off += cout;
    }
    /* head */
    double *h1 = (double *)malloc(sizeof(double) * (size_t)B * F);
    double *h1d = (double *)malloc(sizeof(double) * (size_t)B * F);
    double loss = 0.0;
    for (int b = 0; b < B; ++b) {
        const double *feat = act[4] + (int64_t)b * fin;
        double out = params[off_f2b];
        for (int f = 0; f < F; ++f) {
            double acc = params[off_f1b + f];
            for (int i = 0; i < fin; ++i) acc += params[off_f1w + (int64_t)f * fin + i] * feat[i];
            double r = acc > 0.0 ? acc : 0.0;
            h1[b * F + f] = acc;
            double dr = r;
            if (train && keep) dr = keep[b * F + f] ? r / (1.0 - p) : 0.0;
            h1d[b * F + f] = dr;
            out += params[off_f2w + f] * dr;
        }
        logits[b] = out;
        if (labels) {
            /* BCE with logits, numerically stable form */
            double z = out, t = labels[b];
            loss += (z > 0 ? z : 0.0) - z * t + log1p(exp(-fabs(z)));
        }
    }
    if (labels) loss /= (double)B;

    if (grads && train && labels) {
        memset(grads, 0, sizeof(double) * (size_t)n_params_of(d));
        if (gmag) memset(gmag, 0, sizeof(double) * (size_t)n_params_of(d));
        double *dfeat = (double *)calloc((size_t)nact[4], sizeof(double));
        for (int b = 0; b < B; ++b) {
            double sig = 1.0 / (1.0 + exp(-logits[b]));
            double dz = (sig - labels[b]) / (double)B;
            grads[off_f2b] += dz;
            if (gmag) gmag[off_f2b] += fabs(dz);
            const double *feat = act[4] + (int64_t)b * fin;
            for (int f = 0; f < F; ++f) {
                grads[off_f2w + f] += dz * h1d[b * F + f];
                if (gmag) gmag[off_f2w + f] += fabs(dz * h1d[b * F + f]);
                double dh = dz * params[off_f2w + f];
                if (train && keep) dh = keep[b * F + f] ? dh / (1.0 - p) : 0.0;
                if (h1[b * F + f] <= 0.0) dh = 0.0;
                grads[off_f1b + f] += dh;
                if (gmag) gmag[off_f1b + f] += fabs(dh);
                for (int i = 0; i < fin; ++i) {
                    grads[off_f1w + (int64_t)f * fin + i] += dh * feat[i];
                    if (gmag) gmag[off_f1w + (int64_t)f * fin + i] += fabs(dh * feat[i]);
                    dfeat[(int64_t)b * fin + i] += dh * params[off_f1w + (int64_t)f * fin + i];
                }
            }
        }
        double *dnext = dfeat;   /* gradient w.r.t. act[l+1] */
        for (int l = 3; l >= 0; --l) {
            const int D = dims[l][0], H = dims[l][1], W = dims[l][2], cin = dims[l][3], cout = d->C[l];
            const int D2 = dims[l + 1][0], H2 = dims[l + 1][1], W2 = dims[l + 1][2];
            const int64_t n = npos[l] * cout;
            double *dz = (double *)calloc((size_t)n, sizeof(double));
            /* pool + ReLU backward: gradient to the (first) arg-max, if positive */
            for (int b = 0; b < B; ++b)
                for (int z = 0; z < D2; ++z)
                    for (int y = 0; y < H2; ++y)
                        for (int xw = 0; xw < W2; ++xw)
                            for (int c = 0; c < cout; ++c) {
                                double m = -INFINITY;
                                int64_t arg = -1;
                                for (int ddz = 0; ddz < 2; ++ddz)
                                    for (int ddy = 0; ddy < 2; ++ddy)
                                        for (int ddx = 0; ddx < 2; ++ddx) {
                                            int64_t q = (((int64_t)b * D + 2 * z + ddz) * H + 2 * y + ddy) * W +
                                                        2 * xw + ddx;
                                            double v = zpre[l][q * cout + c];
                                            if (v < 0.0) v = 0.0;
                                            if (v > m) { m = v; arg = q; }
                                        }
                                double gout = dnext[((((int64_t)b * D2 + z) * H2 + y) * W2 + xw) * cout + c];
                                if (zpre[l][arg * cout + c] > 0.0) dz[arg * cout + c] += gout;
                            }
            /* batch-norm backward */
            const double *g = params + off_g[l];
            double *dy = (double *)malloc(sizeof(double) * (size_t)n);
            for (int c = 0; c < cout; ++c) {
                double sdz = 0.0, sdzh = 0.0, mdz = 0.0, mdzh = 0.0;
                for (int64_t q = 0; q < npos[l]; ++q) {
                    sdz += dz[q * cout + c];
                    sdzh += dz[q * cout + c] * yhat[l][q * cout + c];
                    mdz += fabs(dz[q * cout + c]);
                    mdzh += fabs(dz[q * cout + c] * yhat[l][q * cout + c]);
                }
                grads[off_b[l] + c] = sdz;
                grads[off_g[l] + c] = sdzh;
                if (gmag) {
                    gmag[off_b[l] + c] = mdz;
                    gmag[off_g[l] + c] = mdzh;
                }
                const double N = (double)npos[l];
                for (int64_t q = 0; q < npos[l]; ++q) {
                    double v = g[c] * rstd[l][c] / N * (N * dz[q * cout + c] - sdz - yhat[l][q * cout + c] * sdzh);
                    dy[q * cout + c] = bf16_storage ? round_bf16(v) : v;
                }
            }
            /* conv backward: weights and input */
            double *dw = grads + off_w[l];
            double *mw = gmag ? gmag + off_w[l] : NULL;
            const double *w = params + off_w[l];
            double *din = (double *)calloc((size_t)nact[l], sizeof(double));
            for (int b = 0; b < B; ++b)
                for (int z = 0; z < D; ++z)
                    for (int y = 0; y < H; ++y)
                        for (int xw = 0; xw < W; ++xw)
                            for (int co = 0; co < cout; ++co) {
                                double go = dy[((((int64_t)b * D + z) * H + y) * W + xw) * cout + co];
                                if (go == 0.0) continue;
                                for (int kz = 0; kz < 3; ++kz)
                                    for (int ky = 0; ky < 3; ++ky)
                                        for (int kx = 0; kx < 3; ++kx) {
                                            int zz = z + kz - 1, yy = y + ky - 1, xx = xw + kx - 1;
                                            if (zz < 0 || zz >= D || yy < 0 || yy >= H || xx < 0 || xx >= W)
                                                continue;
                                            int64_t ii = ((((int64_t)b * D + zz) * H + yy) * W + xx) * cin;
                                            int64_t wi = ((int64_t)co * 27 + (kz * 3 + ky) * 3 + kx) * cin;
                                            for (int ci = 0; ci < cin; ++ci) {
                                                dw[wi + ci] += go * act[l][ii + ci];
                                                if (mw) mw[wi + ci] += fabs(go * act[l][ii + ci]);
                                                din[ii + ci] += go * w[wi + ci];
                                            }
                                        }
                            }
            free(dz);
            free(dy);
            free(dnext);
            dnext = din;
        }
        free(dnext);
    }
    for (int s = 0; s < 5; ++s) free(act[s]);
    for (int l = 0; l < 4; ++l) {
        free(yconv[l]); free(yhat[l]); free(zpre[l]); free(mean[l]); free(rstd[l]);
    }
    free(h1);
    free(h1d);
    return loss;
}

double orc_cnn_forward_backward_ex(const orc_cnn_dims *d, const double *params, const double *x,
                                   const double *labels, const uint8_t *keep, double p, int train,
                                   double *run_mean, double *run_var, double *logits, double *grads,
                                   int bf16_storage)
{
    return orc_cnn_forward_backward_mag(d, params, x, labels, keep, p, train, run_mean, run_var, logits, grads,
                                        bf16_storage, NULL);
}

double orc_cnn_forward_backward(const orc_cnn_dims *d, const double *params, const double *x,
                                const double *labels, const uint8_t *keep, double p, int train,
                                double *run_mean, double *run_var, double *logits, double *grads)
{
    return orc_cnn_forward_backward_ex(d, params, x, labels, keep, p, train, run_mean, run_var, logits, grads, 0);
}

/* One Adam step (Kingma & Ba 2015) on n parameters, step t >= 1:
 * m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void orc_adam(int64_t n, double *p, const double *g, double *m, double *v, int t, double lr, double b1,
              double b2, double eps)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
