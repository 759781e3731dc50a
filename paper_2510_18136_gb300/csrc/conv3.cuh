// 3x3x3 convolution with zero padding 1 of a channels-last volume x[b][z][y][x][CI]
// with weights w[CO][27][CI] (tap = (dz * 3 + dy) * 3 + dx), FP32 output y[voxel][CO],
// on the tensor cores (BF16 mma.m16n8k16, FP32 accumulation) from a halo tile in
// shared memory.
//
// A CTA keeps all the weights in shared memory and walks output bricks of 2 x 8 x 8
// voxels (128 rows of the GEMM, the brick's voxels in (z, y, x) order).  Each brick's
// 4 x 10 x 10 input halo is copied once with cp.async (zero outside the volume, double
// buffered when it fits); the A fragments of every tap come straight from the halo
// through ldmatrix with one row address per lane (a tap is only an offset), so the K
// loop has no index arithmetic.  Row pitches of CI + 8 and 27 CI + 8 elements keep the
// ldmatrix rows on distinct banks.  With part set, the epilogue also leaves the
// brick's column sums of y and y^2 (fixed order) for batch-norm statistics.
#pragma once

#include "gemm.cuh"

namespace nsfrb {
namespace conv3 {

using bf16 = __nv_bfloat16;

constexpr int BZ = 2, BY = 8, BX = 8;                                  // output brick
constexpr int HZ = BZ + 2, HY = BY + 2, HX = BX + 2, HV = HZ * HY * HX;   // its halo
constexpr int kThreads = 128;                                          // 4 warps x 32 rows

template <int CI, int CO>
struct Shape {
    static constexpr int HP = CI + 8;         // halo row pitch (elements)
    static constexpr int WK = 27 * CI + 8;    // weight row pitch (elements)
    static constexpr size_t w_bytes = sizeof(bf16) * CO * WK;
    static constexpr size_t h_bytes = sizeof(bf16) * HV * HP;
    static constexpr size_t r_bytes = sizeof(float) * 4 * CO * 2;
    static constexpr size_t smem(int nbuf) { return w_bytes + nbuf * h_bytes + r_bytes; }
};

// Bricks are numbered b-major, then z, y, x: brick (b, zb, yb, xb) covers
// z in [2 zb, 2 zb + 2), y in [8 yb, 8 yb + 8), x in [8 xb, 8 xb + 8).  D % 2 = H % 8 = W % 8 = 0.
template <int CI, int CO, int NBUF>
__global__ void __launch_bounds__(kThreads) conv3_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ w,
                                                         float *__restrict__ y, float *__restrict__ part, int D,
                                                         int H, int W, int n_bricks) {
    using S = Shape<CI, CO>;
    constexpr int NI = CO / 8;
    static_assert(CI % 16 == 0 && CO % 16 == 0, "channels must be multiples of 16");
    extern __shared__ __align__(128) unsigned char smem[];
    bf16 *s_w = reinterpret_cast<bf16 *>(smem);
    bf16 *s_h = reinterpret_cast<bf16 *>(smem + S::w_bytes);
    float (*red)[CO][2] = reinterpret_cast<float (*)[CO][2]>(smem + S::w_bytes + NBUF * S::h_bytes);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nxb = W / BX, nyb = H / BY, nzb = D / BZ;

    // all weights, once per CTA
    for (int c = tid; c < CO * (27 * CI / 8); c += kThreads) {
        const int co = c / (27 * CI / 8), kc = (c - co * (27 * CI / 8)) * 8;
        gemm::cp_async16(s_w + co * S::WK + kc, w + static_cast<int64_t>(co) * 27 * CI + kc, true);
    }
    gemm::cp_async_commit();

    auto brick_origin = [&](int bi, int &b, int &z0, int &y0, int &x0) {
        const int xb = bi % nxb, t1 = bi / nxb, yb = t1 % nyb, t2 = t1 / nyb, zb = t2 % nzb;
        b = t2 / nzb;
        z0 = zb * BZ;
        y0 = yb * BY;
        x0 = xb * BX;
    };
    auto load_halo = [&](int bi, int nb) {
        int b, z0, y0, x0;
        brick_origin(bi, b, z0, y0, x0);
        bf16 *dst = s_h + static_cast<size_t>(nb) * HV * S::HP;
        for (int c = tid; c < HV * (CI / 8); c += kThreads) {
            const int hv = c / (CI / 8), cc = (c - hv * (CI / 8)) * 8;
            const int hz = hv / (HY * HX), hy = (hv / HX) % HY, hx = hv % HX;
            const int zz = z0 + hz - 1, yy = y0 + hy - 1, xx = x0 + hx - 1;
            const bool ok = zz >= 0 && zz < D && yy >= 0 && yy < H && xx >= 0 && xx < W;
            const bf16 *src = ok ? x + ((((static_cast<int64_t>(b) * D + zz) * H + yy) * W + xx) * CI + cc) : x;
            gemm::cp_async16(dst + hv * S::HP + cc, src, ok);
        }
        gemm::cp_async_commit();
    };

    // this lane's A rows (tile rows 32 warp + 16 i + (lane & 7) + 8 ((lane >> 3) & 1)) as halo
    // voxels of the centre tap, and the k offset of its ldmatrix row
    int hrow[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int r = 32 * warp + 16 * i + (lane & 7) + 8 * ((lane >> 3) & 1);
        const int bz = r >> 6, by = (r >> 3) & 7, bx = r & 7;
        hrow[i] = ((bz + 1) * HY + by + 1) * HX + bx + 1;
    }
    const int ka = 8 * (lane >> 4);
    const int jb = lane >> 3, rb = lane & 7;
    const int g = lane >> 2, tg = lane & 3;

    if (blockIdx.x < n_bricks) load_halo(blockIdx.x, 0);
    int it = 0;
    for (int bi = blockIdx.x; bi < n_bricks; bi += gridDim.x, ++it) {
        const int nb = (NBUF == 2) ? (it & 1) : 0;
        if (NBUF == 2 && bi + static_cast<int>(gridDim.x) < n_bricks) {
            load_halo(bi + gridDim.x, nb ^ 1);
            gemm::cp_async_wait<1>();
        } else {
            gemm::cp_async_wait<0>();
        }
        __syncthreads();
        const bf16 *hb = s_h + static_cast<size_t>(nb) * HV * S::HP;

        float acc[2][NI][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < NI; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

#pragma unroll 1
        for (int tap = 0; tap < 27; ++tap) {
            const int toff = ((tap / 9 - 1) * HY + (tap / 3) % 3 - 1) * HX + tap % 3 - 1;
#pragma unroll
            for (int kk = 0; kk < CI; kk += 16) {
                uint32_t af[2][4], bfr[NI][2];
#pragma unroll
                for (int i = 0; i < 2; ++i)
                    gemm::ldsm_x4(af[i][0], af[i][1], af[i][2], af[i][3], hb + (hrow[i] + toff) * S::HP + kk + ka);
#pragma unroll
                for (int jn = 0; jn < NI; jn += 2)
                    gemm::ldsm_x4(bfr[jn][0], bfr[jn][1], bfr[jn + 1][0], bfr[jn + 1][1],
                                  s_w + (jn * 8 + rb + 8 * (jb >> 1)) * S::WK + tap * CI + kk + 8 * (jb & 1));
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int jn = 0; jn < NI; ++jn) gemm::mma_bf16(acc[i][jn], af[i], bfr[jn][0], bfr[jn][1]);
            }
        }

        // epilogue: tile row r -> voxel of the brick
        int b, z0, y0, x0;
        brick_origin(bi, b, z0, y0, x0);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = 32 * warp + 16 * i + g + 8 * h;
                const int64_t p = ((static_cast<int64_t>(b) * D + z0 + (r >> 6)) * H + y0 + ((r >> 3) & 7)) * W + x0 +
                                  (r & 7);
#pragma unroll
                for (int jn = 0; jn < NI; ++jn)
                    *reinterpret_cast<float2 *>(y + p * CO + jn * 8 + 2 * tg) =
                        make_float2(acc[i][jn][2 * h], acc[i][jn][2 * h + 1]);
            }
        if (part != nullptr) {
            // column sums (and of squares) over the 128 rows: lanes, then the 4 warps, fixed order
#pragma unroll
            for (int jn = 0; jn < NI; ++jn)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    float cs = 0.0f, cq = 0.0f;
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float v = acc[i][jn][2 * h + e];
                            cs += v;
                            cq += v * v;
                        }
#pragma unroll
                    for (int o = 4; o < 32; o <<= 1) {
                        cs += __shfl_xor_sync(0xffffffffu, cs, o);
                        cq += __shfl_xor_sync(0xffffffffu, cq, o);
                    }
                    if (g == 0) {
                        red[warp][jn * 8 + 2 * tg + e][0] = cs;
                        red[warp][jn * 8 + 2 * tg + e][1] = cq;
                    }
                }
            __syncthreads();
            for (int col = tid; col < CO; col += kThreads) {
                float cs = 0.0f, cq = 0.0f;
                for (int q = 0; q < 4; ++q) {
                    cs += red[q][col][0];
                    cq += red[q][col][1];
                }
                part[(static_cast<int64_t>(bi) * 2) * CO + col] = cs;
                part[(static_cast<int64_t>(bi) * 2 + 1) * CO + col] = cq;
            }
        }
        // every read of this halo buffer (and of red) is done before it is refilled
        __syncthreads();
        if (NBUF == 1 && bi + static_cast<int>(gridDim.x) < n_bricks) load_halo(bi + gridDim.x, 0);
    }
    gemm::cp_async_wait<0>();
}

}  // namespace conv3
}  // namespace nsfrb

namespace nsfrb {
namespace conv3 {

// Weight gradient of the same convolution: dW[co][tap][ci] = sum_voxels dy[v][co] x[v + tap][ci].
// A CTA takes a contiguous range of bricks; per brick the input halo and the brick's 128 x CO
// tile of dy are staged in shared memory (double buffered) and 8 warps each accumulate up to 4
// taps (warp w: taps w, w + 8, w + 16, w + 24) in registers: A = dy^T (ldmatrix.trans of the dy
// tile), B = the halo shifted by the tap (ldmatrix.trans with one row address per lane).  The
// CTA writes its sums to partial[blockIdx.x][CO][27 CI]; wgrad_reduce_kernel adds the CTAs'
// partials in order.
constexpr int kWgThreads = 256;

template <int CI, int CO>
struct WgShape {
    static constexpr int HP = CI + 8, YP = CO + 8;
    static constexpr size_t h_bytes = sizeof(bf16) * HV * HP;
    static constexpr size_t y_bytes = sizeof(bf16) * BZ * BY * BX * YP;
    static constexpr size_t smem = 2 * (h_bytes + y_bytes);
    static constexpr int ACC = 4 * (CO / 16) * (CI / 8) * 4;   // accumulator floats per lane
};

template <int CI, int CO>
__global__ void __launch_bounds__(kWgThreads, 1) conv3_wgrad_kernel(const bf16 *__restrict__ x,
                                                                    const bf16 *__restrict__ dy,
                                                                    float *__restrict__ partial, int D, int H, int W,
                                                                    int n_bricks) {
    using S = WgShape<CI, CO>;
    constexpr int MI = CO / 16, NI = CI / 8;
    static_assert(CI % 16 == 0 && CO % 16 == 0, "channels must be multiples of 16");
    extern __shared__ __align__(128) unsigned char smem[];
    bf16 *s_h = reinterpret_cast<bf16 *>(smem);                      // [2][HV][HP]
    bf16 *s_y = reinterpret_cast<bf16 *>(smem + 2 * S::h_bytes);     // [2][128][YP]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nxb = W / BX, nyb = H / BY, nzb = D / BZ;
    const int bi0 = static_cast<int>(static_cast<int64_t>(blockIdx.x) * n_bricks / gridDim.x);
    const int bi1 = static_cast<int>(static_cast<int64_t>(blockIdx.x + 1) * n_bricks / gridDim.x);

    auto brick_origin = [&](int bi, int &b, int &z0, int &y0, int &x0) {
        const int xb = bi % nxb, t1 = bi / nxb, yb = t1 % nyb, t2 = t1 / nyb, zb = t2 % nzb;
        b = t2 / nzb;
        z0 = zb * BZ;
        y0 = yb * BY;
        x0 = xb * BX;
    };
    auto load = [&](int bi, int nb) {
        int b, z0, y0, x0;
        brick_origin(bi, b, z0, y0, x0);
        bf16 *hd = s_h + static_cast<size_t>(nb) * HV * S::HP;
        for (int c = tid; c < HV * (CI / 8); c += kWgThreads) {
            const int hv = c / (CI / 8), cc = (c - hv * (CI / 8)) * 8;
            const int hz = hv / (HY * HX), hy = (hv / HX) % HY, hx = hv % HX;
            const int zz = z0 + hz - 1, yy = y0 + hy - 1, xx = x0 + hx - 1;
            const bool ok = zz >= 0 && zz < D && yy >= 0 && yy < H && xx >= 0 && xx < W;
            const bf16 *src = ok ? x + ((((static_cast<int64_t>(b) * D + zz) * H + yy) * W + xx) * CI + cc) : x;
            gemm::cp_async16(hd + hv * S::HP + cc, src, ok);
        }
        bf16 *yd = s_y + static_cast<size_t>(nb) * 128 * S::YP;
        for (int c = tid; c < 128 * (CO / 8); c += kWgThreads) {
            const int r = c / (CO / 8), cc = (c - r * (CO / 8)) * 8;
            const int64_t p = ((static_cast<int64_t>(b) * D + z0 + (r >> 6)) * H + y0 + ((r >> 3) & 7)) * W + x0 +
                              (r & 7);
            gemm::cp_async16(yd + r * S::YP + cc, dy + p * CO + cc, true);
        }
        gemm::cp_async_commit();
    };

    // the ldmatrix.trans row of this lane for B at step s: brick voxel 16 s + (lane & 7) +
    // 8 ((lane >> 3) & 1), as a halo voxel of the centre tap (A rows: 16 s + (lane & 7) + 8 (lane >> 4))
    const int jb = lane >> 3, rb = lane & 7;
    int hr[8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int r = 16 * s + rb + 8 * (jb & 1);
        hr[s] = (((r >> 6) + 1) * HY + ((r >> 3) & 7) + 1) * HX + (r & 7) + 1;
    }
    int toff[4];
    bool tok[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int tap = warp + 8 * q;
        tok[q] = tap < 27;
        const int t = tok[q] ? tap : 0;
        toff[q] = ((t / 9 - 1) * HY + (t / 3) % 3 - 1) * HX + t % 3 - 1;
    }
    float acc[4][MI][NI][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < MI; ++i)
#pragma unroll
            for (int j = 0; j < NI; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[q][i][j][e] = 0.0f;

    if (bi0 < bi1) load(bi0, 0);
    int it = 0;
    for (int bi = bi0; bi < bi1; ++bi, ++it) {
        const int nb = it & 1;
        if (bi + 1 < bi1) {
            load(bi + 1, nb ^ 1);
            gemm::cp_async_wait<1>();
        } else {
            gemm::cp_async_wait<0>();
        }
        __syncthreads();
        const bf16 *hb = s_h + static_cast<size_t>(nb) * HV * S::HP;
        const bf16 *yb = s_y + static_cast<size_t>(nb) * 128 * S::YP;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int kk = 16 * s;
            uint32_t af[MI][4];
#pragma unroll
            for (int i = 0; i < MI; ++i)
                gemm::ldsm_x4_t(af[i][0], af[i][1], af[i][2], af[i][3],
                                yb + (kk + rb + 8 * (jb >> 1)) * S::YP + 16 * i + 8 * (jb & 1));
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!tok[q]) continue;
                uint32_t bfr[NI][2];
#pragma unroll
                for (int jn = 0; jn < NI; jn += 2)
                    gemm::ldsm_x4_t(bfr[jn][0], bfr[jn][1], bfr[jn + 1][0], bfr[jn + 1][1],
                                    hb + (hr[s] + toff[q]) * S::HP + jn * 8 + 8 * (jb >> 1));
#pragma unroll
                for (int i = 0; i < MI; ++i)
#pragma unroll
                    for (int jn = 0; jn < NI; ++jn) gemm::mma_bf16(acc[q][i][jn], af[i], bfr[jn][0], bfr[jn][1]);
            }
        }
        __syncthreads();
    }

    // partial[blockIdx.x][co][tap * CI + ci]
    const int g = lane >> 2, tg = lane & 3;
    float *out = partial + static_cast<int64_t>(blockIdx.x) * CO * 27 * CI;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (!tok[q]) continue;
        const int tap = warp + 8 * q;
#pragma unroll
        for (int i = 0; i < MI; ++i)
#pragma unroll
            for (int jn = 0; jn < NI; ++jn)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int co = 16 * i + g + 8 * h;
                    *reinterpret_cast<float2 *>(out + static_cast<int64_t>(co) * 27 * CI + tap * CI + jn * 8 + 2 * tg) =
                        make_float2(acc[q][i][jn][2 * h], acc[q][i][jn][2 * h + 1]);
                }
    }
}

// out[i] = sum over c = 0..n_part-1 of partial[c][i], in that order.
__global__ void wgrad_reduce_kernel(const float *__restrict__ partial, int n_part, int64_t n, float *__restrict__ out) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float s = 0.0f;
        for (int c = 0; c < n_part; ++c) s += partial[static_cast<int64_t>(c) * n + i];
        out[i] = s;
    }
}

}  // namespace conv3
}  // namespace nsfrb
