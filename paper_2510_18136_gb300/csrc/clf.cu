// Candidate classifier of arXiv 2510.18136 Sec. 2.3 (convolutional blocks
// with batch normalisation, ReLU and max-pooling, a small fully connected
// head with dropout, one logit, binary cross-entropy, Adam), trained and run
// on the GPU by the kernels in this file.
//
// Layout: activations channels-last [B][D][H][W][C] (D = time), BF16 between
// layers; convolutions are GEMMs over the (never stored) im2col rows, gathered
// tile by tile from the activations, with BF16 tensor-core MMA and FP32
// accumulation (gemm.cuh); batch-norm statistics, the head, the loss and Adam
// run in FP32.  The flat FP32 parameter vector has the layout
//   for l = 0..3: W_l[C_l][27][C_{l-1}], gamma_l[C_l], beta_l[C_l];
//   fc1_w[F][Fin], fc1_b[F], fc2_w[F], fc2_b[1]
// (tap k = (kz*3 + ky)*3 + kx; Fin = D/16 * H/16 * W/16 * C_3).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "conv3.cuh"
#include "conv3_tc.cuh"
#include "gemm.cuh"
#include "nsfrb_debug.h"
#include "plan_internal.h"

namespace nsfrb {
namespace clf {

using bf16 = __nv_bfloat16;
constexpr int kTB = 256;

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC 2011): ten rounds of two 32x32 multiplies
// with the published multipliers and Weyl key increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// ------------------------------------------------------------------ kernels


// Final reduction in FP64: mean, rstd (biased variance), running statistics.
// Per channel c (one CTA of kFinThreads): the sums over the nblk block partials of part[b][0][c]
// and part[b][1][c] in FP64, as thread-strided sums followed by a fixed shared-memory tree
// (the same order every run).
constexpr int kFinThreads = 256;
__device__ __forceinline__ void channel_sums(const float *__restrict__ part, int nblk, int C, int c, double &s,
                                             double &q) {
    __shared__ double sh[2][kFinThreads];
    double a = 0.0, b2 = 0.0;
    for (int b = threadIdx.x; b < nblk; b += kFinThreads) {
        a += part[static_cast<int64_t>(b) * 2 * C + c];
        b2 += part[static_cast<int64_t>(b) * 2 * C + C + c];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b2;
    __syncthreads();
    for (int o = kFinThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    s = sh[0][0];
    q = sh[1][0];
}

__global__ void __launch_bounds__(kFinThreads) bn_finish_kernel(const float *__restrict__ part, int nblk, int C,
                                                                int64_t P, float eps, float momentum,
                                                                int update_running, float *__restrict__ mean,
                                                                float *__restrict__ rstd, float *__restrict__ run_mean,
                                                                float *__restrict__ run_var) {
    const int c = blockIdx.x;
    double s, q;
    channel_sums(part, nblk, C, c, s, q);
    if (threadIdx.x != 0) return;
    const double mu = s / static_cast<double>(P);
    double var = q / static_cast<double>(P) - mu * mu;
    if (var < 0.0) var = 0.0;
    mean[c] = static_cast<float>(mu);
    rstd[c] = static_cast<float>(1.0 / sqrt(var + eps));
    if (update_running) {
        const double unb = P > 1 ? var * static_cast<double>(P) / static_cast<double>(P - 1) : 0.0;
        run_mean[c] = static_cast<float>((1.0 - momentum) * run_mean[c] + momentum * mu);
        run_var[c] = static_cast<float>((1.0 - momentum) * run_var[c] + momentum * unb);
    }
}

// Backward of max-pool, ReLU and batch norm over pooling windows.  The gradient at the
// batch-norm output, dz, is dpool at the window's arg-max voxel when the pre-ReLU value
// there is positive, else 0; it is recomputed here from (dpool, arg, y) rather than stored.
// Window w of the pooled volume [B][D/2][H/2][W/2] and its voxel q (dz, dy, dx bits).
struct PoolGeom {
    int D, H, W, C;
    gemm::FastDiv fW2, fH2, fD2, fC;
};

inline PoolGeom make_pool_geom(int D, int H, int W, int C) {
    PoolGeom pg;
    pg.D = D;
    pg.H = H;
    pg.W = W;
    pg.C = C;
    pg.fW2 = gemm::make_fastdiv(W / 2);
    pg.fH2 = gemm::make_fastdiv(H / 2);
    pg.fD2 = gemm::make_fastdiv(D / 2);
    pg.fC = gemm::make_fastdiv(C);
    return pg;
}

__device__ __forceinline__ int64_t window_voxel(int64_t w, int q, const PoolGeom &g) {
    const int W2 = g.W / 2, H2 = g.H / 2, D2 = g.D / 2;
    const int wi = static_cast<int>(w);
    const int t1 = gemm::fdiv(wi, g.fW2), t2 = gemm::fdiv(t1, g.fH2), b = gemm::fdiv(t2, g.fD2);
    const int x2 = wi - t1 * W2, y2 = t1 - t2 * H2, z2 = t2 - b * D2;
    return ((static_cast<int64_t>(b) * g.D + 2 * z2 + (q >> 2)) * g.H + 2 * y2 + ((q >> 1) & 1)) * g.W + 2 * x2 +
           (q & 1);
}

// Per-block partial sums over windows [blockIdx.x * wpb, ...) of dz and dz * yhat per channel
// (only the arg-max voxel of a window can carry dz), reduced over the block's threads in a
// fixed order: part[block][0][c], part[block][1][c].
__global__ void __launch_bounds__(kTB) bn_bwd_pool_partial_kernel(const float *__restrict__ dpool,
                                                                  const uint8_t *__restrict__ arg,
                                                                  const float *__restrict__ y,
                                                                  const float *__restrict__ mean,
                                                                  const float *__restrict__ rstd,
                                                                  const float *__restrict__ gamma,
                                                                  const float *__restrict__ beta, int64_t n_win,
                                                                  int wpb, PoolGeom pg, float *__restrict__ part) {
    __shared__ float sh[2][kTB];
    const int C = pg.C;
    const int c = threadIdx.x % C, lanes = kTB / C, ro = threadIdx.x / C;
    float s = 0.0f, q = 0.0f;
    if (ro < lanes) {
        const float mu = mean[c], rs = rstd[c], ga = gamma[c], be = beta[c];
        const int64_t w0 = static_cast<int64_t>(blockIdx.x) * wpb, w1 = min(n_win, w0 + wpb);
        for (int64_t w = w0 + ro; w < w1; w += lanes) {
            const int64_t i = w * C + c;
            const int a = arg[i];
            const float yh = (y[window_voxel(w, a, pg) * C + c] - mu) * rs;
            const float dzv = (ga * yh + be > 0.0f) ? dpool[i] : 0.0f;
            s += dzv;
            q += dzv * yh;
        }
    }
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = q;
    __syncthreads();
    // rows ro = 0..lanes-1 of channel c sit at threadIdx c + ro * C: fixed halving tree over ro
    for (int n = lanes; n > 1;) {
        const int half = (n + 1) / 2;
        if (ro + half < n) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + half * C];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + half * C];
        }
        n = half;
        __syncthreads();
    }
    if (ro == 0) {
        part[static_cast<int64_t>(blockIdx.x) * 2 * C + c] = sh[0][c];
        part[static_cast<int64_t>(blockIdx.x) * 2 * C + C + c] = sh[1][c];
    }
}

// dy = gamma * rstd / N * (N dz - sum dz - yhat * sum(dz yhat)) for the 8 voxels of every
// window, as BF16 for the GEMMs.
__global__ void bn_bwd_pool_apply_kernel(const float *__restrict__ dpool, const uint8_t *__restrict__ arg,
                                         const float *__restrict__ y, const float *__restrict__ mean,
                                         const float *__restrict__ rstd, const float *__restrict__ gamma,
                                         const float *__restrict__ beta, const float *__restrict__ dgamma,
                                         const float *__restrict__ dbeta, int64_t n_win, int64_t P, PoolGeom pg,
                                         bf16 *__restrict__ dy) {
    const int C = pg.C;
    const float N = static_cast<float>(P);
    const int64_t total = n_win * C;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int w = gemm::fdiv(static_cast<int>(i), pg.fC);   // n_win * C < 2^31 (checked at creation)
        const int c = static_cast<int>(i) - w * C;
        const int a = arg[i];
        const float dp = dpool[i];
        const float mu = mean[c], rs = rstd[c], ga = gamma[c], be = beta[c], db = dbeta[c], dg = dgamma[c];
        const int64_t v0 = window_voxel(w, 0, pg);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t pos = v0 + (static_cast<int64_t>((q >> 2)) * pg.H + ((q >> 1) & 1)) * pg.W + (q & 1);
            const float yh = (y[pos * C + c] - mu) * rs;
            const float dzv = (q == a && ga * yh + be > 0.0f) ? dp : 0.0f;
            dy[pos * C + c] = __float2bfloat16_rn(ga * rs / N * (N * dzv - db - yh * dg));
        }
    }
}

// Inference: the running statistics take the place of the batch statistics.
__global__ void bn_eval_kernel(const float *__restrict__ run_mean, const float *__restrict__ run_var, int C,
                               float eps, float *__restrict__ mean, float *__restrict__ rstd) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    mean[c] = run_mean[c];
    rstd[c] = 1.0f / sqrtf(run_var[c] + eps);
}

// BN -> ReLU -> 2x2x2 max-pool; writes the pooled BF16 activation and the
// arg-max (first in (dz, dy, dx) order) for the backward pass.
__global__ void bn_relu_pool_kernel(const float *__restrict__ y, const float *__restrict__ mean,
                                    const float *__restrict__ rstd, const float *__restrict__ gamma,
                                    const float *__restrict__ beta, int64_t n_win, PoolGeom pg,
                                    bf16 *__restrict__ out, uint8_t *__restrict__ arg) {
    const int C = pg.C;
    const int64_t total = n_win * C;   // < 2^31 (checked at creation)
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int w = gemm::fdiv(static_cast<int>(i), pg.fC);
        const int c = static_cast<int>(i) - w * C;
        const float g = gamma[c], be = beta[c], mu = mean[c], rs = rstd[c];
        const int64_t v0 = window_voxel(w, 0, pg);
        float m = -INFINITY;
        int a = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t pos = v0 + (static_cast<int64_t>(q >> 2) * pg.H + ((q >> 1) & 1)) * pg.W + (q & 1);
            float v = g * ((y[pos * C + c] - mu) * rs) + be;
            v = fmaxf(v, 0.0f);
            if (v > m) {
                m = v;
                a = q;
            }
        }
        out[i] = __float2bfloat16_rn(m);
        arg[i] = static_cast<uint8_t>(a);
    }
}



// dbeta = sum dz, dgamma = sum dz * yhat (written into the gradient vector).
__global__ void __launch_bounds__(kFinThreads) bn_bwd_finish_kernel(const float *__restrict__ part, int nblk, int C,
                                                                    float *__restrict__ dgamma,
                                                                    float *__restrict__ dbeta) {
    const int c = blockIdx.x;
    double s, q;
    channel_sums(part, nblk, C, c, s, q);
    if (threadIdx.x != 0) return;
    dbeta[c] = static_cast<float>(s);
    dgamma[c] = static_cast<float>(q);
}


// Head forward: features (BF16) -> FC1 -> ReLU -> dropout -> FC2 -> logit;
// loss terms.  One block per sample.
__global__ void head_fwd_kernel(const bf16 *__restrict__ feat_bf, int Fin, int F, const float *__restrict__ w1,
                                const float *__restrict__ b1, const float *__restrict__ w2,
                                const float *__restrict__ b2, int train, float p, uint2 key, uint32_t step,
                                const float *__restrict__ labels, float *__restrict__ feat, float *__restrict__ h1,
                                float *__restrict__ h1d, float *__restrict__ logit, float *__restrict__ loss_terms) {
    extern __shared__ float sfeat[];   // [Fin] then [F]
    const int b = blockIdx.x;
    for (int i = threadIdx.x; i < Fin; i += blockDim.x) {
        const float v = __bfloat162float(feat_bf[static_cast<int64_t>(b) * Fin + i]);
        sfeat[i] = v;
        feat[static_cast<int64_t>(b) * Fin + i] = v;
    }
    __syncthreads();
    float *sh = sfeat + Fin;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int f = warp; f < F; f += nw) {
        float acc = 0.0f;
        for (int i = lane; i < Fin; i += 32) acc += w1[static_cast<int64_t>(f) * Fin + i] * sfeat[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const float pre = acc + b1[f];
            float r = fmaxf(pre, 0.0f);
            if (train && p > 0.0f) {
                const uint4 u = philox4x32_10(make_uint4(static_cast<uint32_t>(b * F + f), step, 0u, 0u), key);
                const float uu = static_cast<float>(u.x >> 8) * (1.0f / 16777216.0f);
                r = (uu >= p) ? r / (1.0f - p) : 0.0f;
            }
            h1[b * F + f] = pre;
            h1d[b * F + f] = r;
            sh[f] = r;
        }
    }
    __syncthreads();
    if (warp == 0) {
        float acc = 0.0f;
        for (int f = lane; f < F; f += 32) acc += w2[f] * sh[f];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const float z = acc + b2[0];
            logit[b] = z;
            if (labels) {
                const float t = labels[b];
                loss_terms[b] = fmaxf(z, 0.0f) - z * t + log1pf(expf(-fabsf(z)));
            }
        }
    }
}

// Head backward (one block): FC2, dropout, ReLU, FC1 gradients and the
// gradient of the pooled features.  Small: B x F x Fin.
__global__ void head_bwd_kernel(int B, int Fin, int F, const float *__restrict__ feat,
                                const float *__restrict__ h1, const float *__restrict__ h1d,
                                const float *__restrict__ logit, const float *__restrict__ labels,
                                const float *__restrict__ w1, const float *__restrict__ w2, float p, uint2 key,
                                uint32_t step, float *__restrict__ dh1, float *__restrict__ g_b1,
                                float *__restrict__ g_w2, float *__restrict__ g_b2) {
    // dh1[b][f] and the FC2 gradients (the FC1 weight gradient: head_dw1_kernel)
    for (int i = threadIdx.x; i < B * F; i += blockDim.x) {
        const int b = i / F, f = i % F;
        const float dz = (1.0f / (1.0f + expf(-logit[b])) - labels[b]) / static_cast<float>(B);
        float d = dz * w2[f];
        if (p > 0.0f) {
            const uint4 u = philox4x32_10(make_uint4(static_cast<uint32_t>(b * F + f), step, 0u, 0u), key);
            const float uu = static_cast<float>(u.x >> 8) * (1.0f / 16777216.0f);
            d = (uu >= p) ? d / (1.0f - p) : 0.0f;
        }
        if (h1[i] <= 0.0f) d = 0.0f;
        dh1[i] = d;
    }
    __syncthreads();
    for (int f = threadIdx.x; f < F; f += blockDim.x) {
        float sw = 0.0f, sb = 0.0f;
        for (int b = 0; b < B; ++b) {
            const float dz = (1.0f / (1.0f + expf(-logit[b])) - labels[b]) / static_cast<float>(B);
            sw += dz * h1d[b * F + f];
            sb += dh1[b * F + f];
        }
        g_w2[f] = sw;
        g_b1[f] = sb;
    }
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int b = 0; b < B; ++b) s += (1.0f / (1.0f + expf(-logit[b])) - labels[b]) / static_cast<float>(B);
        g_b2[0] = s;
    }
}

// FC1 weight gradient g_w1[f][k] = sum_b dh1[b][f] feat[b][k] (b ascending), one output per thread.
__global__ void head_dw1_kernel(int B, int Fin, int F, const float *__restrict__ feat, const float *__restrict__ dh1,
                                float *__restrict__ g_w1) {
    const int64_t n = static_cast<int64_t>(F) * Fin;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int f = static_cast<int>(i / Fin), k = static_cast<int>(i - static_cast<int64_t>(f) * Fin);
        float s = 0.0f;
        for (int b = 0; b < B; ++b) s += dh1[b * F + f] * feat[static_cast<int64_t>(b) * Fin + k];
        g_w1[i] = s;
    }
}

// Gradient of the pooled features: dfeat[b][k] = sum_f dh1[b][f] w1[f][k].
__global__ void head_dfeat_kernel(int B, int Fin, int F, const float *__restrict__ dh1, const float *__restrict__ w1,
                                  float *__restrict__ dfeat) {
    const int64_t total = static_cast<int64_t>(B) * Fin;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int b = static_cast<int>(i / Fin), k = static_cast<int>(i % Fin);
        float s = 0.0f;
        for (int f = 0; f < F; ++f) s += dh1[b * F + f] * w1[static_cast<int64_t>(f) * Fin + k];
        dfeat[i] = s;
    }
}

__global__ void sum_kernel(const float *__restrict__ v, int n, float scale, float *__restrict__ out) {
    __shared__ float sh[kTB];
    float s = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0] * scale;
}

// Adam (Kingma & Ba 2015) on the FP32 master parameters.
__global__ void adam_kernel(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// BF16 copies of conv weights W[co][k][ci] and of the flipped, transposed
// weights Wf[ci][k'][co] = W[co][26 - k'][ci] used for the input gradient.
__global__ void weights_bf16_kernel(const float *__restrict__ w, int Co, int Ci, bf16 *__restrict__ wb,
                                    bf16 *__restrict__ wf) {
    const int64_t total = static_cast<int64_t>(Co) * 27 * Ci;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int ci = static_cast<int>(i % Ci);
        const int k = static_cast<int>((i / Ci) % 27);
        const int co = static_cast<int>(i / (static_cast<int64_t>(Ci) * 27));
        const bf16 v = __float2bfloat16_rn(w[i]);
        wb[i] = v;
        wf[(static_cast<int64_t>(ci) * 27 + (26 - k)) * Co + co] = v;
    }
}

// Cutouts around candidates: out[i][z][y][x][k] (BF16) = mean over the b
// samples of time bin z of cube[(r0 + y) * nx + c0 + x][k][ts + z*b + j] / scale,
// zero outside the image and the window.  b = max(1, ceil((w + smax) / (D/2)))
// so that the pulse's dispersed extent fills at most half the cutout; the
// window is centred on t_idx + (w + smax) / 2.
__global__ void cutout_kernel(const void *__restrict__ cube, int dtype, int ny, int nx, int n_sub, int n_t,
                              const float *__restrict__ sigma, float sigma_default,
                              const CandRec *__restrict__ cand, int n, const int32_t *__restrict__ smax,
                              const int32_t *__restrict__ widths, int D, int H, int W, bf16 *__restrict__ out) {
    const int64_t per = static_cast<int64_t>(D) * H * W * n_sub;
    const int64_t total = per * n;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int k = static_cast<int>(i % n_sub);
        int64_t r = i / n_sub;
        const int x = static_cast<int>(r % W);
        const int y = static_cast<int>((r / W) % H);
        const int z = static_cast<int>((r / (static_cast<int64_t>(W) * H)) % D);
        const int c = static_cast<int>(r / (static_cast<int64_t>(W) * H * D));
        const CandRec cr = cand[c];
        const int w = widths[cr.w_idx];
        const int sm = smax[cr.dm_idx];
        const int span = w + sm;
        int bin = (span + D / 2 - 1) / (D / 2);
        if (bin < 1) bin = 1;
        const int ts = cr.t_idx + span / 2 - (D * bin) / 2;
        const int row = cr.row - H / 2 + y, col = cr.col - W / 2 + x;
        float v = 0.0f;
        if (row >= 0 && row < ny && col >= 0 && col < nx) {
            const int64_t pix = static_cast<int64_t>(row) * nx + col;
            const int64_t base = (pix * n_sub + k) * n_t;
            float acc = 0.0f;
            for (int j = 0; j < bin; ++j) {
                const int t = ts + z * bin + j;
                if (t < 0 || t >= n_t) continue;
                if (dtype == 0)
                    acc += static_cast<const float *>(cube)[base + t];
                else {
                    const unsigned short u = static_cast<const unsigned short *>(cube)[base + t];
                    acc += (dtype == 1) ? __uint_as_float(static_cast<uint32_t>(u) << 16)
                                        : __half2float(__ushort_as_half(u));
                }
            }
            const int64_t pc = static_cast<int64_t>(cr.row) * nx + cr.col;
            const float sg = sigma ? sigma[pc] : sigma_default;
            v = acc / static_cast<float>(bin) / (sg / sqrtf(static_cast<float>(n_sub)));
        }
        out[i] = __float2bfloat16_rn(v);
    }
}

inline int grid_for(int64_t n) { return static_cast<int>(std::min<int64_t>((n + kTB - 1) / kTB, 152 * 32)); }

}  // namespace clf
}  // namespace nsfrb

// ============================================================================ object

struct nsfrb_clf_s {
    nsfrb_clf_config cfg{};
    int dims[5][4] = {};      // D, H, W, C entering conv l (row 4: pooled output of the last block)
    int64_t off_w[4] = {}, off_g[4] = {}, off_b[4] = {}, off_f1w = 0, off_f1b = 0, off_f2w = 0, off_f2b = 0;
    int64_t n_params = 0;
    int Fin = 0;
    int64_t step = 0;           // training steps done (dropout counter, Adam t - 1)
    // device buffers
    float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    float *run_mean = nullptr, *run_var = nullptr;   // [sum C_l]
    __nv_bfloat16 *wb[4] = {}, *wf[4] = {};
    __nv_bfloat16 *act[5] = {};                       // act[0] unused (caller input)
    uint8_t *arg[4] = {};
    float *y[4] = {};
    float *mean[4] = {}, *rstd[4] = {};
    __nv_bfloat16 *dyb = nullptr;
    float *dact = nullptr, *part = nullptr;
    float *feat = nullptr, *h1 = nullptr, *h1d = nullptr, *logit = nullptr, *loss_terms = nullptr, *loss = nullptr;
    float *dh1 = nullptr;
    float *labels_zero = nullptr;
    int64_t zmax = 0, dact_elems = 0;
    int part_blocks = 0;
    int max_smem = 0, n_sm = 0;   // device properties for the convolution kernels
    float *wpart = nullptr;       // per-CTA weight-gradient partials
    int64_t wpart_elems = 0;
    nsfrb_status latched = NSFRB_OK;
};

namespace {

using namespace nsfrb;
using namespace nsfrb::clf;

nsfrb_status clf_cuda(nsfrb_clf_s *c, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return NSFRB_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    if (c && c->latched == NSFRB_OK) c->latched = NSFRB_ECUDA;
    return NSFRB_ECUDA;
}

nsfrb_status clf_fail(nsfrb_status st, const std::string &msg) {
    set_error(msg);
    return st;
}

// Device word of error bits latched by the kernels (after the loss in the same allocation).
int *clf_err(nsfrb_clf_s *c) { return reinterpret_cast<int *>(c->loss + 1); }

constexpr int kWinPerBlock = 64;     // pooling windows per block of the batch-norm backward partials

// C[M][N] = A[M][K] B[N][K]^T; with gx.x set, A is the im2col matrix of gx (gathered).
// With part set, also the column sums of C and of C^2 per 128-row tile: part[tile][2][N].
constexpr int kGemmRows = 128;
template <int G>
nsfrb_status gemm_nt_g(int64_t M, int N, int K, const bf16 *A, const bf16 *B, float *C, gemm::Gather gx,
                       cudaStream_t s, float *part = nullptr) {
    if (N <= 32) {
        const dim3 g2(static_cast<unsigned>((M + 127) / 128), static_cast<unsigned>((N + 31) / 32), 1);
        gemm::gemm_kernel<128, 32, false, G>
            <<<g2, gemm::kThreads, 0, s>>>(static_cast<int>(M), N, K, A, K, B, K, C, N, 1, gx, part);
    } else {
        const dim3 grid(static_cast<unsigned>((M + 127) / 128), static_cast<unsigned>((N + 63) / 64), 1);
        gemm::gemm_kernel<128, 64, false, G>
            <<<grid, gemm::kThreads, 0, s>>>(static_cast<int>(M), N, K, A, K, B, K, C, N, 1, gx, part);
    }
    return cudaGetLastError() == cudaSuccess ? NSFRB_OK : NSFRB_ECUDA;
}

// C[M][N] (zeroed here) = A[K][M]^T B[K][N] with split-K over K; with gx.x set, B is the
// im2col matrix of gx (gathered).
// Tiles and split-K count of the TN GEMM: tile rows follow M (the output channels: 32 or 64 in
// the network), wide tiles along N, about 4 CTAs per SM of 152.
inline int tn_split(int M, int N, int64_t K, int &bm, int &mt, int &nt) {
    bm = M <= 32 ? 32 : (M <= 64 ? 64 : 128);
    const int bn = bm == 128 ? 64 : 128;
    mt = (M + bm - 1) / bm;
    nt = (N + bn - 1) / bn;
    const int64_t k_steps = (K + gemm::BK - 1) / gemm::BK;
    return std::max(1, static_cast<int>(std::min<int64_t>(k_steps, std::max<int64_t>(1, 4 * 152 / (mt * nt)))));
}

// With a workspace of wpart_elems floats that holds split x M x N, the splits' partials are summed in
// split order (reproducible); otherwise they are added atomically.
template <int G>
nsfrb_status gemm_tn_g(int M, int N, int64_t K, const bf16 *A, const bf16 *B, float *C, gemm::Gather gx,
                       cudaStream_t s, float *wpart = nullptr, int64_t wpart_elems = 0) {
    int bm, mt, nt;
    const int split = tn_split(M, N, K, bm, mt, nt);
    const dim3 grid(mt, nt, split);
    float *part = (wpart && static_cast<int64_t>(split) * M * N <= wpart_elems) ? wpart : nullptr;
    if (!part && cudaMemsetAsync(C, 0, sizeof(float) * static_cast<size_t>(M) * N, s) != cudaSuccess)
        return NSFRB_ECUDA;
    if (bm == 32)
        gemm::gemm_kernel<32, 128, true, G><<<grid, gemm::kThreads, 0, s>>>(M, N, static_cast<int>(K), A, M, B, N, C,
                                                                             N, split, gx, part);
    else if (bm == 64)
        gemm::gemm_kernel<64, 128, true, G><<<grid, gemm::kThreads, 0, s>>>(M, N, static_cast<int>(K), A, M, B, N, C,
                                                                             N, split, gx, part);
    else
        gemm::gemm_kernel<128, 64, true, G><<<grid, gemm::kThreads, 0, s>>>(M, N, static_cast<int>(K), A, M, B, N, C,
                                                                             N, split, gx, part);
    if (part) {
        const int64_t n = static_cast<int64_t>(M) * N;
        conv3::wgrad_reduce_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(part, split, n, C);
    }
    return cudaGetLastError() == cudaSuccess ? NSFRB_OK : NSFRB_ECUDA;
}

// 3x3x3 convolution y = conv(x, w) by the halo-tile kernel when the channel pair has an
// instance, the volume divides into 2 x 8 x 8 bricks and the shared memory fits (two halo
// buffers if possible, else one).  Returns false when it does not apply (nothing launched).
template <int CI, int CO, int NBUF>
bool conv3_try(const bf16 *x, const bf16 *w, float *y, float *part, int B, int D, int H, int W, int max_smem,
               int n_sm, cudaStream_t s, cudaError_t &err) {
    const size_t smem = conv3::Shape<CI, CO>::smem(NBUF);
    if (smem > static_cast<size_t>(max_smem)) return false;
    static int blocks_per_sm = 0;   // per instance: attribute set and occupancy read once
    if (blocks_per_sm == 0) {
        err = cudaFuncSetAttribute(conv3::conv3_kernel<CI, CO, NBUF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(smem));
        if (err == cudaSuccess)
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, conv3::conv3_kernel<CI, CO, NBUF>,
                                                                conv3::kThreads, smem);
        if (err != cudaSuccess) return true;
        blocks_per_sm = std::max(blocks_per_sm, 1);
    }
    const int n_bricks = B * (D / conv3::BZ) * (H / conv3::BY) * (W / conv3::BX);
    const int grid = std::min(n_bricks, blocks_per_sm * n_sm);
    conv3::conv3_kernel<CI, CO, NBUF><<<grid, conv3::kThreads, smem, s>>>(x, w, y, part, D, H, W, n_bricks);
    err = cudaGetLastError();
    return true;
}

// Resident CTAs per SM of an instance (0 if its shared memory does not fit).
template <int CI, int CO, int NBUF>
int conv3_occupancy(int max_smem) {
    static int occ = -1;
    if (occ < 0) {
        const size_t smem = conv3::Shape<CI, CO>::smem(NBUF);
        occ = 0;
        if (smem <= static_cast<size_t>(max_smem) &&
            cudaFuncSetAttribute(conv3::conv3_kernel<CI, CO, NBUF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem)) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, conv3::conv3_kernel<CI, CO, NBUF>, conv3::kThreads,
                                                          smem) != cudaSuccess)
            occ = 0;
        cudaGetLastError();
    }
    return occ;
}

// 3x3x3 convolution on tcgen05 when the volume divides into 1 x 16 x 8 bricks and the shared
// memory fits.  The grid is the CTAs that shared memory lets reside on every SM, at most
// 512 / (the CTA's tensor-memory columns) so that no CTA waits for tensor memory.  Returns
// false when it does not apply (nothing launched).
template <int CI, int CO>
bool conv3_tc_try(const bf16 *x, const bf16 *w, float *y, float *part, int B, int D, int H, int W, int max_smem,
                  int n_sm, int *d_err, cudaStream_t s, cudaError_t &err, int stall = 0) {
    using S = conv3tc::Shape<CI, CO>;
    if (H % conv3tc::BY || W % conv3tc::BX || W < 16 || D < 4) return false;
    static int blocks_per_sm = 0;   // per instance: attribute set and residency computed once; -1: not usable
    if (blocks_per_sm == 0) {
        blocks_per_sm = -1;
        int dev = 0, sm_smem = 0, reserved = 0;
        cudaGetDevice(&dev);
        if (S::smem <= static_cast<size_t>(max_smem) &&
            cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) == cudaSuccess &&
            cudaFuncSetAttribute(conv3tc::conv3_tc_kernel<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(S::smem)) == cudaSuccess) {
            cudaFuncAttributes fa{};
            if (cudaFuncGetAttributes(&fa, conv3tc::conv3_tc_kernel<CI, CO>) == cudaSuccess) {
                const int by_smem = sm_smem / static_cast<int>(S::smem + reserved);
                const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;   // allocation unit: 256 per warp
                const int by_regs = 65536 / (warp_regs * (conv3tc::kThreads / 32));
                blocks_per_sm = std::min(std::min(by_smem, by_regs), static_cast<int>(512u / S::cols));
                if (blocks_per_sm < 1) blocks_per_sm = -1;
            }
        }
        cudaGetLastError();
    }
    if (blocks_per_sm < 1) return false;
    const int n_bricks = B * D * (H / conv3tc::BY) * (W / conv3tc::BX);
    const int grid = std::min(n_bricks, blocks_per_sm * n_sm);
    conv3tc::conv3_tc_kernel<CI, CO><<<grid, conv3tc::kThreads, S::smem, s>>>(x, w, y, part, D, H, W, n_bricks, d_err,
                                                                             stall);
    err = cudaGetLastError();
    return true;
}

// Two halo buffers unless one buffer keeps more CTAs (warps) resident per SM.
template <int CI, int CO>
bool conv3_pair(const bf16 *x, const bf16 *w, float *y, float *part, int B, int D, int H, int W, int max_smem,
                int n_sm, cudaStream_t s, cudaError_t &err) {
    const int o2 = conv3_occupancy<CI, CO, 2>(max_smem), o1 = conv3_occupancy<CI, CO, 1>(max_smem);
    if (o2 > 0 && o2 >= o1) return conv3_try<CI, CO, 2>(x, w, y, part, B, D, H, W, max_smem, n_sm, s, err);
    if (o1 > 0) return conv3_try<CI, CO, 1>(x, w, y, part, B, D, H, W, max_smem, n_sm, s, err);
    return false;
}

// Weight gradient dW = sum_voxels dy x(tap) by the halo-tile kernel (into the partial workspace,
// then a fixed-order sum into dw) when the channel pair keeps <= 128 accumulators per lane, the
// volume divides into bricks and the shared memory fits; false when it does not apply.
template <int CI, int CO>
bool wgrad_pair(const bf16 *x, const bf16 *dy, float *wpart, int64_t wpart_elems, float *dw, int B, int D, int H,
                int W, int max_smem, int n_sm, cudaStream_t s, cudaError_t &err) {
    using S = conv3::WgShape<CI, CO>;
    if (S::ACC > 128 || S::smem > static_cast<size_t>(max_smem)) return false;
    const int n_bricks = B * (D / conv3::BZ) * (H / conv3::BY) * (W / conv3::BX);
    const int grid = std::min(n_bricks, n_sm);
    const int64_t n = static_cast<int64_t>(CO) * 27 * CI;
    if (static_cast<int64_t>(grid) * n > wpart_elems) return false;
    static bool attr = false;
    if (!attr) {
        err = cudaFuncSetAttribute(conv3::conv3_wgrad_kernel<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(S::smem));
        if (err != cudaSuccess) return true;
        attr = true;
    }
    conv3::conv3_wgrad_kernel<CI, CO><<<grid, conv3::kWgThreads, S::smem, s>>>(x, dy, wpart, D, H, W, n_bricks);
    conv3::wgrad_reduce_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(wpart, grid, n, dw);
    err = cudaGetLastError();
    return true;
}

bool wgrad_launch(int CI, int CO, const bf16 *x, const bf16 *dy, float *wpart, int64_t wpart_elems, float *dw, int B,
                  int D, int H, int W, int max_smem, int n_sm, cudaStream_t s, cudaError_t &err) {
    err = cudaSuccess;
    if (D % conv3::BZ || H % conv3::BY || W % conv3::BX) return false;
#define NSFRB_WGRAD(A, Bc)                                                                                 \
    if (CI == A && CO == Bc)                                                                               \
        return wgrad_pair<A, Bc>(x, dy, wpart, wpart_elems, dw, B, D, H, W, max_smem, n_sm, s, err);
    NSFRB_WGRAD(16, 16) NSFRB_WGRAD(16, 32) NSFRB_WGRAD(16, 64)
    NSFRB_WGRAD(32, 16) NSFRB_WGRAD(32, 32) NSFRB_WGRAD(64, 16)
#undef NSFRB_WGRAD
    return false;
}

// 3x3x3 convolution by the tcgen05 kernel if it applies, else by the mma.sync halo kernel;
// false when neither does (nothing launched).  paths: bit 0 allows the halo kernel, bit 1 the
// tcgen05 kernel; bit 2 (tests) runs the tcgen05 kernel with stalled producers, so that its
// waits time out.  *used tells which ran (1 or 2).
bool conv3_launch(int CI, int CO, const bf16 *x, const bf16 *w, float *y, float *part, int B, int D, int H, int W,
                  int max_smem, int n_sm, int *d_err, cudaStream_t s, cudaError_t &err, int paths = 3,
                  int *used = nullptr) {
    err = cudaSuccess;
    if (used) *used = 2;
    const int stall = (paths & 4) ? 1 : 0;
#define NSFRB_CONV3_TC(A, Bc)                                                                          \
    if (CI == A && CO == Bc &&                                                                          \
        conv3_tc_try<A, Bc>(x, w, y, part, B, D, H, W, max_smem, n_sm, d_err, s, err, stall))           \
        return true;
    if (paths & 6) {
        NSFRB_CONV3_TC(16, 16) NSFRB_CONV3_TC(16, 32) NSFRB_CONV3_TC(16, 64)
        NSFRB_CONV3_TC(32, 16) NSFRB_CONV3_TC(32, 32) NSFRB_CONV3_TC(32, 64) NSFRB_CONV3_TC(64, 16)
    }
#undef NSFRB_CONV3_TC
    if (used) *used = 1;
    if (!(paths & 1)) return false;
    if (D % conv3::BZ || H % conv3::BY || W % conv3::BX) return false;
#define NSFRB_CONV3(A, Bc)                                                                               \
    if (CI == A && CO == Bc) return conv3_pair<A, Bc>(x, w, y, part, B, D, H, W, max_smem, n_sm, s, err);
    NSFRB_CONV3(16, 16) NSFRB_CONV3(16, 32) NSFRB_CONV3(16, 64)
    NSFRB_CONV3(32, 16) NSFRB_CONV3(32, 32) NSFRB_CONV3(32, 64)
    NSFRB_CONV3(64, 16) NSFRB_CONV3(64, 32) NSFRB_CONV3(64, 64)
#undef NSFRB_CONV3
    return false;
}

nsfrb_status gemm_nt(int64_t M, int N, int K, const bf16 *A, const bf16 *B, float *C, cudaStream_t s) {
    return gemm_nt_g<0>(M, N, K, A, B, C, gemm::Gather{}, s);
}
nsfrb_status gemm_tn(int M, int N, int64_t K, const bf16 *A, const bf16 *B, float *C, cudaStream_t s) {
    return gemm_tn_g<0>(M, N, K, A, B, C, gemm::Gather{}, s);
}

// Forward of the conv blocks and the head; keeps everything the backward needs.
nsfrb_status forward(nsfrb_clf_s *c, const bf16 *x, const float *labels, int B, int train, cudaStream_t s) {
    const nsfrb_clf_config &cf = c->cfg;
    const bf16 *in = x;
    int64_t rs = 0;
    for (int l = 0; l < 4; ++l) {
        const int D = c->dims[l][0], H = c->dims[l][1], W = c->dims[l][2], Ci = c->dims[l][3], Co = cf.c[l];
        const int64_t P = static_cast<int64_t>(B) * D * H * W;
        // training: the convolution also leaves the per-tile (128-row) channel sums of y and y^2
        cudaError_t ce;
        if (conv3_launch(Ci, Co, in, c->wb[l], c->y[l], train ? c->part : nullptr, B, D, H, W, c->max_smem, c->n_sm,
                         clf_err(c), s, ce)) {
            if (ce != cudaSuccess) return clf_cuda(c, ce, "conv3");
        } else if (gemm_nt_g<1>(P, Co, 27 * Ci, nullptr, c->wb[l], c->y[l], gemm::make_gather(in, D, H, W, Ci), s,
                                train ? c->part : nullptr) != NSFRB_OK) {
            return clf_cuda(c, cudaGetLastError(), "conv gemm");
        }
        if (train) {
            const int nblk = static_cast<int>((P + kGemmRows - 1) / kGemmRows);
            bn_finish_kernel<<<Co, kFinThreads, 0, s>>>(c->part, nblk, Co, P, 1e-5f, cf.bn_momentum, 1, c->mean[l],
                                                        c->rstd[l], c->run_mean + rs, c->run_var + rs);
        } else {
            bn_eval_kernel<<<(Co + 63) / 64, 64, 0, s>>>(c->run_mean + rs, c->run_var + rs, Co, 1e-5f, c->mean[l],
                                                         c->rstd[l]);
        }
        const int64_t npool = P / 8 * Co;
        bn_relu_pool_kernel<<<grid_for(npool), kTB, 0, s>>>(c->y[l], c->mean[l], c->rstd[l], c->params + c->off_g[l],
                                                            c->params + c->off_b[l], P / 8, make_pool_geom(D, H, W, Co),
                                                            c->act[l + 1], c->arg[l]);
        in = c->act[l + 1];
        rs += Co;
    }
    const uint2 key = make_uint2(static_cast<uint32_t>(cf.seed), static_cast<uint32_t>(cf.seed >> 32));
    const size_t hs = sizeof(float) * (c->Fin + cf.f);
    head_fwd_kernel<<<B, kTB, hs, s>>>(c->act[4], c->Fin, cf.f, c->params + c->off_f1w, c->params + c->off_f1b,
                                       c->params + c->off_f2w, c->params + c->off_f2b, train, cf.dropout, key,
                                       static_cast<uint32_t>(c->step), labels, c->feat, c->h1, c->h1d, c->logit,
                                       c->loss_terms);
    if (labels) sum_kernel<<<1, kTB, 0, s>>>(c->loss_terms, B, 1.0f / static_cast<float>(B), c->loss);
    return clf_cuda(c, cudaGetLastError(), "forward");
}

nsfrb_status backward(nsfrb_clf_s *c, const bf16 *x, const float *labels, int B, cudaStream_t s) {
    const nsfrb_clf_config &cf = c->cfg;
    const uint2 key = make_uint2(static_cast<uint32_t>(cf.seed), static_cast<uint32_t>(cf.seed >> 32));
    head_bwd_kernel<<<1, kTB, 0, s>>>(B, c->Fin, cf.f, c->feat, c->h1, c->h1d, c->logit, labels,
                                      c->params + c->off_f1w, c->params + c->off_f2w, cf.dropout, key,
                                      static_cast<uint32_t>(c->step), c->dh1, c->grads + c->off_f1b,
                                      c->grads + c->off_f2w, c->grads + c->off_f2b);
    head_dw1_kernel<<<grid_for(static_cast<int64_t>(cf.f) * c->Fin), kTB, 0, s>>>(B, c->Fin, cf.f, c->feat, c->dh1,
                                                                                c->grads + c->off_f1w);
    head_dfeat_kernel<<<grid_for(static_cast<int64_t>(B) * c->Fin), kTB, 0, s>>>(B, c->Fin, cf.f, c->dh1,
                                                                               c->params + c->off_f1w, c->dact);
    for (int l = 3; l >= 0; --l) {
        const int D = c->dims[l][0], H = c->dims[l][1], W = c->dims[l][2], Ci = c->dims[l][3], Co = cf.c[l];
        const int64_t P = static_cast<int64_t>(B) * D * H * W;
        // max-pool, ReLU and batch-norm backward over the pooling windows (dz recomputed)
        const PoolGeom pg = make_pool_geom(D, H, W, Co);
        const int64_t n_win = P / 8;
        const int nblk = static_cast<int>((n_win + kWinPerBlock - 1) / kWinPerBlock);
        bn_bwd_pool_partial_kernel<<<nblk, kTB, 0, s>>>(c->dact, c->arg[l], c->y[l], c->mean[l], c->rstd[l],
                                                        c->params + c->off_g[l], c->params + c->off_b[l], n_win,
                                                        kWinPerBlock, pg, c->part);
        bn_bwd_finish_kernel<<<Co, kFinThreads, 0, s>>>(c->part, nblk, Co, c->grads + c->off_g[l],
                                                        c->grads + c->off_b[l]);
        bn_bwd_pool_apply_kernel<<<grid_for(n_win * Co), kTB, 0, s>>>(
            c->dact, c->arg[l], c->y[l], c->mean[l], c->rstd[l], c->params + c->off_g[l], c->params + c->off_b[l],
            c->grads + c->off_g[l], c->grads + c->off_b[l], n_win, P, pg, c->dyb);
        // weight gradient: dW[co][(k, ci)] = sum_p dy[p][co] col[p][(k, ci)], col gathered from the input
        const bf16 *in = (l == 0) ? x : c->act[l];
        cudaError_t we;
        if (wgrad_launch(Ci, Co, in, c->dyb, c->wpart, c->wpart_elems, c->grads + c->off_w[l], B, D, H, W,
                         c->max_smem, c->n_sm, s, we)) {
            if (we != cudaSuccess) return clf_cuda(c, we, "conv3 weight gradient");
        } else if (gemm_tn_g<2>(Co, 27 * Ci, P, c->dyb, nullptr, c->grads + c->off_w[l],
                                gemm::make_gather(in, D, H, W, Ci), s, c->wpart, c->wpart_elems) != NSFRB_OK) {
            return clf_cuda(c, cudaGetLastError(), "weight gemm");
        }
        if (l > 0) {
            // input gradient: a convolution of dy with the flipped, transposed weights
            cudaError_t ce;
            if (conv3_launch(Co, Ci, c->dyb, c->wf[l], c->dact, nullptr, B, D, H, W, c->max_smem, c->n_sm, clf_err(c), s,
                             ce)) {
                if (ce != cudaSuccess) return clf_cuda(c, ce, "conv3 input gradient");
            } else if (gemm_nt_g<1>(P, Ci, 27 * Co, nullptr, c->wf[l], c->dact, gemm::make_gather(c->dyb, D, H, W, Co),
                                    s) != NSFRB_OK) {
                return clf_cuda(c, cudaGetLastError(), "input gemm");
            }
        }
    }
    return clf_cuda(c, cudaGetLastError(), "backward");
}

void refresh_weights(nsfrb_clf_s *c, cudaStream_t s) {
    for (int l = 0; l < 4; ++l) {
        const int Ci = c->dims[l][3], Co = c->cfg.c[l];
        weights_bf16_kernel<<<grid_for(static_cast<int64_t>(Co) * 27 * Ci), kTB, 0, s>>>(c->params + c->off_w[l], Co,
                                                                                        Ci, c->wb[l], c->wf[l]);
    }
}

}  // namespace

// ============================================================================ C ABI

extern "C" {

nsfrb_status nsfrb_clf_create(const nsfrb_clf_config *cfg, nsfrb_clf_t *out) {
    if (!cfg || !out) return clf_fail(NSFRB_EINVAL, "null argument");
    *out = nullptr;
    const nsfrb_clf_config &c = *cfg;
    if (c.batch < 1 || c.d < 16 || c.h < 16 || c.w < 16 || c.d % 16 || c.h % 16 || c.w % 16)
        return clf_fail(NSFRB_EINVAL, "batch >= 1 and cutout sides multiples of 16 required");
    if (c.c0 < 8 || c.c0 % 8) return clf_fail(NSFRB_EINVAL, "c0 must be a positive multiple of 8");
    for (int l = 0; l < 4; ++l) {
        if (c.c[l] < 8 || c.c[l] % 8 || c.c[l] > kTB) return clf_fail(NSFRB_EINVAL, "channels: multiples of 8 up to 256");
        if (static_cast<int64_t>(c.batch) * c.d * c.h * c.w * std::max(c.c[l], c.c0) >= (int64_t(1) << 31))
            return clf_fail(NSFRB_EINVAL, "batch x cutout voxels x channels must stay below 2^31");
    }
    if (c.f < 1 || c.f > 1024) return clf_fail(NSFRB_EINVAL, "f must be 1..1024");
    if (!(c.dropout >= 0.0f && c.dropout < 1.0f)) return clf_fail(NSFRB_EINVAL, "dropout must be in [0, 1)");
    nsfrb_clf_s *m = new (std::nothrow) nsfrb_clf_s();
    if (!m) return clf_fail(NSFRB_ENOMEM, "classifier allocation");
    m->cfg = c;
    m->dims[0][0] = c.d; m->dims[0][1] = c.h; m->dims[0][2] = c.w; m->dims[0][3] = c.c0;
    for (int l = 0; l < 4; ++l) {
        m->dims[l + 1][0] = m->dims[l][0] / 2;
        m->dims[l + 1][1] = m->dims[l][1] / 2;
        m->dims[l + 1][2] = m->dims[l][2] / 2;
        m->dims[l + 1][3] = c.c[l];
    }
    int64_t o = 0;
    for (int l = 0; l < 4; ++l) {
        m->off_w[l] = o; o += static_cast<int64_t>(c.c[l]) * 27 * m->dims[l][3];
        m->off_g[l] = o; o += c.c[l];
        m->off_b[l] = o; o += c.c[l];
    }
    m->Fin = m->dims[4][0] * m->dims[4][1] * m->dims[4][2] * m->dims[4][3];
    m->off_f1w = o; o += static_cast<int64_t>(c.f) * m->Fin;
    m->off_f1b = o; o += c.f;
    m->off_f2w = o; o += c.f;
    m->off_f2b = o; o += 1;
    m->n_params = o;

    const int B = c.batch;
    int64_t zmax = 0, dact = static_cast<int64_t>(B) * m->Fin, part = 0;
    for (int l = 0; l < 4; ++l) {
        const int64_t P = static_cast<int64_t>(B) * m->dims[l][0] * m->dims[l][1] * m->dims[l][2];
        zmax = std::max(zmax, P * c.c[l]);
        dact = std::max(dact, P * m->dims[l][3]);
        part = std::max(part, ((P + kGemmRows - 1) / kGemmRows) * 2 * c.c[l]);
        part = std::max(part, ((P / 8 + kWinPerBlock - 1) / kWinPerBlock) * 2 * c.c[l]);
    }
    int nc = 0;
    for (int l = 0; l < 4; ++l) nc += c.c[l];
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&m->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, dev);
    }
    bool ok = true;
    auto A = [&](void **p, size_t bytes) {
        if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
    };
    A(reinterpret_cast<void **>(&m->params), sizeof(float) * o);
    A(reinterpret_cast<void **>(&m->grads), sizeof(float) * o);
    A(reinterpret_cast<void **>(&m->adam_m), sizeof(float) * o);
    A(reinterpret_cast<void **>(&m->adam_v), sizeof(float) * o);
    A(reinterpret_cast<void **>(&m->run_mean), sizeof(float) * nc);
    A(reinterpret_cast<void **>(&m->run_var), sizeof(float) * nc);
    for (int l = 0; l < 4; ++l) {
        const int64_t P = static_cast<int64_t>(B) * m->dims[l][0] * m->dims[l][1] * m->dims[l][2];
        const int64_t nw = static_cast<int64_t>(c.c[l]) * 27 * m->dims[l][3];
        A(reinterpret_cast<void **>(&m->wb[l]), sizeof(bf16) * nw);
        A(reinterpret_cast<void **>(&m->wf[l]), sizeof(bf16) * nw);
        A(reinterpret_cast<void **>(&m->y[l]), sizeof(float) * P * c.c[l]);
        A(reinterpret_cast<void **>(&m->arg[l]), P / 8 * c.c[l]);
        A(reinterpret_cast<void **>(&m->act[l + 1]), sizeof(bf16) * (P / 8) * c.c[l]);
        A(reinterpret_cast<void **>(&m->mean[l]), sizeof(float) * c.c[l]);
        A(reinterpret_cast<void **>(&m->rstd[l]), sizeof(float) * c.c[l]);
    }
    A(reinterpret_cast<void **>(&m->dyb), sizeof(bf16) * zmax);
    // per-CTA weight-gradient partials: n_sm CTAs of the halo kernel or the splits of the split-K
    // GEMM, each of Co x 27 Ci floats
    for (int l = 0; l < 4; ++l) {
        const int64_t P = static_cast<int64_t>(B) * m->dims[l][0] * m->dims[l][1] * m->dims[l][2];
        int bm, mt, nt;
        const int split = tn_split(c.c[l], 27 * m->dims[l][3], P, bm, mt, nt);
        m->wpart_elems = std::max<int64_t>(m->wpart_elems, static_cast<int64_t>(std::max(std::max(m->n_sm, 1), split)) *
                                                               c.c[l] * 27 * m->dims[l][3]);
    }
    A(reinterpret_cast<void **>(&m->wpart), sizeof(float) * m->wpart_elems);
    A(reinterpret_cast<void **>(&m->dact), sizeof(float) * dact);
    A(reinterpret_cast<void **>(&m->part), sizeof(float) * std::max<int64_t>(part, 2));
    A(reinterpret_cast<void **>(&m->feat), sizeof(float) * B * m->Fin);
    A(reinterpret_cast<void **>(&m->h1), sizeof(float) * B * c.f);
    A(reinterpret_cast<void **>(&m->h1d), sizeof(float) * B * c.f);
    A(reinterpret_cast<void **>(&m->dh1), sizeof(float) * B * c.f);
    A(reinterpret_cast<void **>(&m->logit), sizeof(float) * B);
    A(reinterpret_cast<void **>(&m->loss_terms), sizeof(float) * B);
    A(reinterpret_cast<void **>(&m->loss), sizeof(float) * 2);   // the loss, then the kernels' error bits
    if (!ok) {
        cudaGetLastError();
        nsfrb_clf_destroy(m);
        return clf_fail(NSFRB_ENOMEM, "classifier device buffers");
    }
    cudaMemset(m->loss, 0, sizeof(float) * 2);
    cudaMemset(m->params, 0, sizeof(float) * o);
    cudaMemset(m->grads, 0, sizeof(float) * o);
    cudaMemset(m->adam_m, 0, sizeof(float) * o);
    cudaMemset(m->adam_v, 0, sizeof(float) * o);
    cudaMemset(m->run_mean, 0, sizeof(float) * nc);
    std::vector<float> ones(nc, 1.0f);
    cudaMemcpy(m->run_var, ones.data(), sizeof(float) * nc, cudaMemcpyHostToDevice);
    refresh_weights(m, 0);
    if (clf_cuda(m, cudaDeviceSynchronize(), "classifier init") != NSFRB_OK) {
        nsfrb_clf_destroy(m);
        return NSFRB_ECUDA;
    }
    *out = m;
    return NSFRB_OK;
}

nsfrb_status nsfrb_clf_n_params(nsfrb_clf_t clf, int64_t *n) {
    if (!clf || !n) return clf_fail(NSFRB_EINVAL, "null argument");
    *n = clf->n_params;
    return NSFRB_OK;
}

nsfrb_status nsfrb_clf_set_params(nsfrb_clf_t clf, const float *h_params) {
    if (!clf || !h_params) return clf_fail(NSFRB_EINVAL, "null argument");
    nsfrb_status st = clf_cuda(clf, cudaMemcpy(clf->params, h_params, sizeof(float) * clf->n_params,
                                                cudaMemcpyHostToDevice), "set params");
    if (st != NSFRB_OK) return st;
    refresh_weights(clf, 0);
    return clf_cuda(clf, cudaDeviceSynchronize(), "set params");
}

nsfrb_status nsfrb_clf_get_params(nsfrb_clf_t clf, float *h_params) {
    if (!clf || !h_params) return clf_fail(NSFRB_EINVAL, "null argument");
    return clf_cuda(clf, cudaMemcpy(h_params, clf->params, sizeof(float) * clf->n_params, cudaMemcpyDeviceToHost),
                    "get params");
}

nsfrb_status nsfrb_clf_get_grads(nsfrb_clf_t clf, float *h_grads) {
    if (!clf || !h_grads) return clf_fail(NSFRB_EINVAL, "null argument");
    return clf_cuda(clf, cudaMemcpy(h_grads, clf->grads, sizeof(float) * clf->n_params, cudaMemcpyDeviceToHost),
                    "get grads");
}

static int clf_nc(const nsfrb_clf_s *c) { return c->cfg.c[0] + c->cfg.c[1] + c->cfg.c[2] + c->cfg.c[3]; }

nsfrb_status nsfrb_clf_get_bn_stats(nsfrb_clf_t clf, float *h_run_mean, float *h_run_var) {
    if (!clf) return clf_fail(NSFRB_EINVAL, "null argument");
    const size_t b = sizeof(float) * clf_nc(clf);
    nsfrb_status st = NSFRB_OK;
    if (h_run_mean) st = clf_cuda(clf, cudaMemcpy(h_run_mean, clf->run_mean, b, cudaMemcpyDeviceToHost), "bn stats");
    if (st == NSFRB_OK && h_run_var)
        st = clf_cuda(clf, cudaMemcpy(h_run_var, clf->run_var, b, cudaMemcpyDeviceToHost), "bn stats");
    return st;
}

nsfrb_status nsfrb_clf_set_bn_stats(nsfrb_clf_t clf, const float *h_run_mean, const float *h_run_var) {
    if (!clf) return clf_fail(NSFRB_EINVAL, "null argument");
    const size_t b = sizeof(float) * clf_nc(clf);
    nsfrb_status st = NSFRB_OK;
    if (h_run_mean) st = clf_cuda(clf, cudaMemcpy(clf->run_mean, h_run_mean, b, cudaMemcpyHostToDevice), "bn stats");
    if (st == NSFRB_OK && h_run_var)
        st = clf_cuda(clf, cudaMemcpy(clf->run_var, h_run_var, b, cudaMemcpyHostToDevice), "bn stats");
    return st;
}

nsfrb_status nsfrb_clf_train_step(nsfrb_clf_t clf, const void *d_x, const float *d_labels, int32_t batch,
                                  int32_t update, float *h_loss, void *stream) {
    if (!clf || !d_x || !d_labels || batch < 1 || batch > clf->cfg.batch)
        return clf_fail(NSFRB_EINVAL, "bad argument");
    if (clf->latched != NSFRB_OK) return clf_fail(clf->latched, "classifier has a latched CUDA error");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bf16 *x = static_cast<const bf16 *>(d_x);
    nsfrb_status st = forward(clf, x, d_labels, batch, 1, s);
    if (st != NSFRB_OK) return st;
    if ((st = backward(clf, x, d_labels, batch, s)) != NSFRB_OK) return st;
    if (update) {
        const nsfrb_clf_config &c = clf->cfg;
        const int t = static_cast<int>(clf->step) + 1;
        const float c1 = 1.0f - powf(c.beta1, static_cast<float>(t));
        const float c2 = 1.0f - powf(c.beta2, static_cast<float>(t));
        adam_kernel<<<grid_for(clf->n_params), kTB, 0, s>>>(clf->n_params, clf->params, clf->grads, clf->adam_m,
                                                            clf->adam_v, c.lr, c.beta1, c.beta2, c.eps, c1, c2);
        refresh_weights(clf, s);
        ++clf->step;
        if ((st = clf_cuda(clf, cudaGetLastError(), "adam")) != NSFRB_OK) return st;
    }
    if (h_loss) {
        float out[2];
        if ((st = clf_cuda(clf, cudaMemcpyAsync(out, clf->loss, sizeof(out), cudaMemcpyDeviceToHost, s),
                           "loss copy")) != NSFRB_OK)
            return st;
        if ((st = clf_cuda(clf, cudaStreamSynchronize(s), "train step")) != NSFRB_OK) return st;
        *h_loss = out[0];
        int bits = 0;
        std::memcpy(&bits, &out[1], sizeof(bits));
        if (bits != 0) {
            clf->latched = NSFRB_ECUDA;
            return clf_fail(NSFRB_ECUDA, "a tensor-core convolution wait timed out");
        }
    }
    return NSFRB_OK;
}

nsfrb_status nsfrb_clf_infer(nsfrb_clf_t clf, const void *d_x, int32_t batch, float *d_logit, void *stream) {
    if (!clf || !d_x || !d_logit || batch < 1 || batch > clf->cfg.batch) return clf_fail(NSFRB_EINVAL, "bad argument");
    if (clf->latched != NSFRB_OK) return clf_fail(clf->latched, "classifier has a latched CUDA error");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    nsfrb_status st = forward(clf, static_cast<const bf16 *>(d_x), nullptr, batch, 0, s);
    if (st != NSFRB_OK) return st;
    return clf_cuda(clf, cudaMemcpyAsync(d_logit, clf->logit, sizeof(float) * batch, cudaMemcpyDeviceToDevice, s),
                    "logits");
}

nsfrb_status nsfrb_clf_cutouts(nsfrb_plan_t plan, const void *d_cube, const float *d_sigma,
                               const nsfrb_candidate *d_cand, int32_t n, int32_t d, int32_t h, int32_t w,
                               void *d_out, void *stream) {
    if (!plan || !d_cube || (n > 0 && (!d_cand || !d_out)) || n < 0 || d < 2 || h < 1 || w < 1)
        return fail(plan, NSFRB_EINVAL, "bad argument");
    if (n == 0) return NSFRB_OK;
    if (!plan->d_smax_w) {
        std::vector<int32_t> t(plan->smax);
        t.insert(t.end(), plan->widths.begin(), plan->widths.end());
        if (cudaMalloc(reinterpret_cast<void **>(&plan->d_smax_w), sizeof(int32_t) * t.size()) != cudaSuccess) {
            cudaGetLastError();
            plan->d_smax_w = nullptr;
            return fail(plan, NSFRB_ENOMEM, "cutout tables");
        }
        nsfrb_status st = cuda_check(plan, cudaMemcpy(plan->d_smax_w, t.data(), sizeof(int32_t) * t.size(),
                                                      cudaMemcpyHostToDevice), "cutout tables");
        if (st != NSFRB_OK) return st;
    }
    const nsfrb_config &c = plan->cfg;
    const int64_t total = static_cast<int64_t>(n) * d * h * w * c.n_sub;
    cutout_kernel<<<grid_for(total), kTB, 0, static_cast<cudaStream_t>(stream)>>>(
        d_cube, c.dtype, c.ny, c.nx, c.n_sub, c.n_t, c.noise_mode == NSFRB_NOISE_KNOWN ? d_sigma : nullptr,
        std::sqrt(static_cast<float>(c.n_sub)), reinterpret_cast<const CandRec *>(d_cand), n, plan->d_smax_w,
        plan->d_smax_w + c.n_dm, d, h, w, static_cast<bf16 *>(d_out));
    return cuda_check(plan, cudaGetLastError(), "cutout launch");
}

nsfrb_status nsfrb_dbg_conv3(int32_t path, int32_t B, int32_t D, int32_t H, int32_t W, int32_t CI, int32_t CO,
                             const void *d_x, const void *d_w, float *d_y, float *d_part, int32_t *d_err,
                             int32_t *h_used, void *stream) {
    if (path < 0 || path > 3 || B < 1 || D < 1 || H < 1 || W < 1 || !d_x || !d_w || !d_y || !d_err)
        return clf_fail(NSFRB_EINVAL, "bad convolution arguments");
    int dev = 0, max_smem = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t ce = cudaSuccess;
    int used = 0;
    const int paths = path == 0 ? 3 : path == 3 ? 4 : path;
    if (!conv3_launch(CI, CO, static_cast<const bf16 *>(d_x), static_cast<const bf16 *>(d_w), d_y, d_part, B, D, H,
                      W, max_smem, n_sm, d_err, static_cast<cudaStream_t>(stream), ce, paths, &used))
        return clf_fail(NSFRB_EINVAL, "no convolution kernel for this shape and path");
    if (ce != cudaSuccess) return clf_cuda(nullptr, ce, "convolution launch");
    if (h_used) *h_used = used;
    return NSFRB_OK;
}

nsfrb_status nsfrb_dbg_gemm(int32_t tn, int32_t M, int32_t N, int32_t K, const void *d_a, const void *d_b,
                            float *d_c, void *stream) {
    if (M < 1 || N < 1 || K < 1 || K % 8 || (tn && (M % 8 || N % 8)) || !d_a || !d_b || !d_c)
        return clf_fail(NSFRB_EINVAL, "bad GEMM shape");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bf16 *a = static_cast<const bf16 *>(d_a), *b = static_cast<const bf16 *>(d_b);
    nsfrb_status st = tn ? gemm_tn(M, N, K, a, b, d_c, s) : gemm_nt(M, N, K, a, b, d_c, s);
    if (st != NSFRB_OK) return clf_fail(st, "GEMM launch");
    return NSFRB_OK;
}

static const char kMagic[8] = {'N', 'S', 'F', 'R', 'B', 'C', 'L', '1'};

nsfrb_status nsfrb_clf_save(nsfrb_clf_t clf, const char *path) {
    if (!clf || !path) return clf_fail(NSFRB_EINVAL, "null argument");
    const int64_t n = clf->n_params;
    const int nc = clf_nc(clf);
    std::vector<float> buf(3 * n + 2 * nc);
    if (clf_cuda(clf, cudaDeviceSynchronize(), "save") != NSFRB_OK) return NSFRB_ECUDA;
    cudaMemcpy(buf.data(), clf->params, sizeof(float) * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(buf.data() + n, clf->adam_m, sizeof(float) * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(buf.data() + 2 * n, clf->adam_v, sizeof(float) * n, cudaMemcpyDeviceToHost);
    cudaMemcpy(buf.data() + 3 * n, clf->run_mean, sizeof(float) * nc, cudaMemcpyDeviceToHost);
    cudaMemcpy(buf.data() + 3 * n + nc, clf->run_var, sizeof(float) * nc, cudaMemcpyDeviceToHost);
    if (clf_cuda(clf, cudaGetLastError(), "save copies") != NSFRB_OK) return NSFRB_ECUDA;
    FILE *fh = std::fopen(path, "wb");
    if (!fh) return clf_fail(NSFRB_EINVAL, "cannot open checkpoint for writing");
    bool ok = std::fwrite(kMagic, 1, 8, fh) == 8 && std::fwrite(&clf->cfg, sizeof(clf->cfg), 1, fh) == 1 &&
              std::fwrite(&n, sizeof(n), 1, fh) == 1 && std::fwrite(&clf->step, sizeof(clf->step), 1, fh) == 1 &&
              std::fwrite(buf.data(), sizeof(float), buf.size(), fh) == buf.size();
    ok = (std::fclose(fh) == 0) && ok;
    return ok ? NSFRB_OK : clf_fail(NSFRB_EINVAL, "checkpoint write failed");
}

nsfrb_status nsfrb_clf_load(nsfrb_clf_t clf, const char *path) {
    if (!clf || !path) return clf_fail(NSFRB_EINVAL, "null argument");
    FILE *fh = std::fopen(path, "rb");
    if (!fh) return clf_fail(NSFRB_EINVAL, "cannot open checkpoint");
    char magic[8];
    nsfrb_clf_config cfg;
    int64_t n = 0, step = 0;
    const int nc = clf_nc(clf);
    bool ok = std::fread(magic, 1, 8, fh) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(&cfg, sizeof(cfg), 1, fh) == 1 && std::fread(&n, sizeof(n), 1, fh) == 1 &&
              std::fread(&step, sizeof(step), 1, fh) == 1 && n == clf->n_params;
    std::vector<float> buf;
    if (ok) {
        buf.resize(3 * n + 2 * nc);
        ok = std::fread(buf.data(), sizeof(float), buf.size(), fh) == buf.size();
    }
    std::fclose(fh);
    if (!ok || std::memcmp(cfg.c, clf->cfg.c, sizeof(cfg.c)) != 0 || cfg.c0 != clf->cfg.c0 || cfg.f != clf->cfg.f)
        return clf_fail(NSFRB_EINVAL, "checkpoint does not match this classifier");
    cudaMemcpy(clf->params, buf.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(clf->adam_m, buf.data() + n, sizeof(float) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(clf->adam_v, buf.data() + 2 * n, sizeof(float) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(clf->run_mean, buf.data() + 3 * n, sizeof(float) * nc, cudaMemcpyHostToDevice);
    cudaMemcpy(clf->run_var, buf.data() + 3 * n + nc, sizeof(float) * nc, cudaMemcpyHostToDevice);
    clf->step = step;
    refresh_weights(clf, 0);
    return clf_cuda(clf, cudaDeviceSynchronize(), "load");
}

void nsfrb_clf_destroy(nsfrb_clf_t clf) {
    if (!clf) return;
    cudaDeviceSynchronize();
    void *ptrs[] = {clf->params, clf->grads, clf->adam_m, clf->adam_v, clf->run_mean, clf->run_var,
                    clf->dyb, clf->wpart, clf->dact, clf->part, clf->feat, clf->h1, clf->h1d, clf->dh1, clf->logit,
                    clf->loss_terms, clf->loss};
    for (void *p : ptrs) cudaFree(p);
    for (int l = 0; l < 4; ++l) {
        cudaFree(clf->wb[l]);
        cudaFree(clf->wf[l]);
        cudaFree(clf->y[l]);
        cudaFree(clf->arg[l]);
        cudaFree(clf->act[l + 1]);
        cudaFree(clf->mean[l]);
        cudaFree(clf->rstd[l]);
    }
    cudaGetLastError();
    delete clf;
}

}  // extern "C"
