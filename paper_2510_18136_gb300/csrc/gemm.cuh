// BF16 tensor-core GEMM with FP32 accumulation for the classifier's
// convolutions (implicit in im2col form) and their gradients.
//
//   NT:  C[M][N]  = A[M][K] * B[N][K]^T      (A, B K-contiguous)
//   TN:  C[M][N] += A[K][M]^T * B[K][N]      (A, B contiguous along M / N; split-K
//                                             partial sums added atomically, or written
//                                             per split to a workspace for an ordered sum)
//
// Tiles of BM x BN x 32 are staged in shared memory with 16-byte cp.async
// (zero-filled outside the matrix, double buffered) and fed to
// mma.m16n8k16 through ldmatrix (.trans for the TN layout).  K must be a
// multiple of 8 and every row start 16-byte aligned.
//
// Implicit convolution (G = 1, 2): the im2col matrix of a channels-last volume
// x[b][z][y][x][c] (3x3x3 taps, zero padding 1, column index tap * C + c with
// tap = (dz * 3 + dy) * 3 + dx) is never stored: the tile loader gathers its 16-byte
// chunks (8 channels of one tap) straight from x, zero-filling taps outside the
// volume.  G = 1 gathers the A rows of an NT product (conv forward / input gradient),
// G = 2 the B operand of a TN product (weight gradient).  C must be a multiple of 8.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

namespace nsfrb {
namespace gemm {

constexpr int BK = 32;
constexpr int kThreads = 128;   // 4 warps

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool pred) {
    const int n = pred ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// TRANS = false: A tile stored [BM][BK+8], B tile [BN][BK+8] (K contiguous)
// TRANS = true:  A tile stored [BK][BM+8], B tile [BK][BN+8] (M / N contiguous)
// Division by an invariant divisor d for 0 <= n < 2^31 (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994, round-up variant):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(n, m) + n) >> l.
struct FastDiv {
    uint32_t m = 1, l = 0;
};
inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f;
    uint32_t l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    f.l = l;
    f.m = static_cast<uint32_t>(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
    return f;
}
__device__ __forceinline__ int fdiv(int n, FastDiv f) {
    return static_cast<int>((__umulhi(static_cast<uint32_t>(n), f.m) + static_cast<uint32_t>(n)) >> f.l);
}

struct Gather {
    const __nv_bfloat16 *x;   // [B][D][H][W][C]
    int D, H, W, C;
    FastDiv fD, fH, fW, fC;
};
inline Gather make_gather(const __nv_bfloat16 *x, int D, int H, int W, int C) {
    Gather g;
    g.x = x;
    g.D = D;
    g.H = H;
    g.W = W;
    g.C = C;
    g.fD = make_fastdiv(D);
    g.fH = make_fastdiv(H);
    g.fW = make_fastdiv(W);
    g.fC = make_fastdiv(C);
    return g;
}

template <int BM, int BN, bool TRANS>
struct Smem {
    static constexpr int A_ELEMS = TRANS ? BK * (BM + 8) : BM * (BK + 8);
    static constexpr int B_ELEMS = TRANS ? BK * (BN + 8) : BN * (BK + 8);
    __nv_bfloat16 a[2][A_ELEMS];
    __nv_bfloat16 b[2][B_ELEMS];
};

// One CTA computes a BM x BN tile of C over the K range [k_lo, k_hi).
template <int BM, int BN, bool TRANS, int G = 0>
__global__ void __launch_bounds__(kThreads) gemm_kernel(int M, int N, int K, const __nv_bfloat16 *__restrict__ A,
                                                        int64_t lda, const __nv_bfloat16 *__restrict__ B,
                                                        int64_t ldb, float *__restrict__ C, int64_t ldc,
                                                        int k_split, Gather gx, float *__restrict__ part) {
    static_assert(G == 0 || (G == 1 && !TRANS) || (G == 2 && TRANS), "gather mode / layout mismatch");
    constexpr int WM = (BN >= 64) ? 2 : 4;    // warps along M
    constexpr int WN = 4 / WM;                // warps along N
    constexpr int TM = BM / WM, TN = BN / WN; // warp tile
    constexpr int MI = TM / 16, NI = TN / 8;
    static_assert(NI % 2 == 0, "warp tile N must be a multiple of 16");
    __shared__ __align__(128) Smem<BM, BN, TRANS> sm;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp % WM, wn = warp / WM;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    // K range of this CTA (split-K along gridDim.z, in whole BK steps)
    const int k_steps = (K + BK - 1) / BK;
    const int per = (k_steps + k_split - 1) / k_split;
    const int ks0 = blockIdx.z * per, ks1 = min(k_steps, ks0 + per);
    if (ks0 >= ks1) return;

    // G = 1: the voxels of this thread's A rows (rows tid/4 + 32 j, chunk column (tid % 4) * 8)
    constexpr int kRowsPer = (G == 1) ? BM * (BK / 8) / kThreads : 1;
    int64_t g_base[kRowsPer];
    int g_z[kRowsPer], g_y[kRowsPer], g_x[kRowsPer];
    if constexpr (G == 1) {
#pragma unroll
        for (int j = 0; j < kRowsPer; ++j) {
            const int gm = m0 + (tid + kThreads * j) / (BK / 8);
            const int v = gm < M ? gm : 0;
            g_x[j] = v % gx.W;
            g_y[j] = (v / gx.W) % gx.H;
            g_z[j] = (v / (gx.W * gx.H)) % gx.D;
            g_base[j] = gm < M ? static_cast<int64_t>(v / (gx.W * gx.H * gx.D)) * gx.D * gx.H * gx.W : -1;
        }
    }
    // G = 2: each thread loads kCPT consecutive chunks of one B row (one voxel); the taps and
    // channels of its chunk columns are fixed for the whole K loop
    constexpr int kCPT = (G == 2) ? BK * (BN / 8) / kThreads : 1;
    static_assert(G != 2 || (BN / 8) % kCPT == 0, "a thread's chunks must lie in one row");
    int g_dz[kCPT], g_dy[kCPT], g_dx[kCPT], g_ci[kCPT];
    bool g_nok[kCPT];
    if constexpr (G == 2) {
#pragma unroll
        for (int j = 0; j < kCPT; ++j) {
            const int gn = n0 + ((tid * kCPT + j) % (BN / 8)) * 8;
            g_nok[j] = gn < N;
            const int tap = fdiv(g_nok[j] ? gn : 0, gx.fC);
            g_ci[j] = (g_nok[j] ? gn : 0) - tap * gx.C;
            g_dz[j] = tap / 9 - 1;
            g_dy[j] = (tap / 3) % 3 - 1;
            g_dx[j] = tap % 3 - 1;
        }
    }

    auto load_tile = [&](int stage, int ks) {
        const int kb = ks * BK;
        if constexpr (G == 1) {
            const int kc = (tid % (BK / 8)) * 8, gk = kb + kc;
            const bool kok = gk < K;
            const int tap = kok ? fdiv(gk, gx.fC) : 0, ci = kok ? gk - tap * gx.C : 0;
            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
#pragma unroll
            for (int j = 0; j < kRowsPer; ++j) {
                const int r = (tid + kThreads * j) / (BK / 8);
                const int zz = g_z[j] + dz, yy = g_y[j] + dy, xx = g_x[j] + dx;
                const bool ok = kok && g_base[j] >= 0 && zz >= 0 && zz < gx.D && yy >= 0 && yy < gx.H && xx >= 0 &&
                                xx < gx.W;
                const __nv_bfloat16 *src =
                    ok ? gx.x + (g_base[j] + (static_cast<int64_t>(zz) * gx.H + yy) * gx.W + xx) * gx.C + ci : gx.x;
                cp_async16(&sm.a[stage][r * (BK + 8) + kc], src, ok);
            }
        } else if constexpr (!TRANS) {
            // A: BM rows x 4 chunks of 8 along K
            for (int c = tid; c < BM * (BK / 8); c += kThreads) {
                const int r = c / (BK / 8), kc = (c % (BK / 8)) * 8;
                const int gm = m0 + r, gk = kb + kc;
                const bool ok = gm < M && gk < K;
                cp_async16(&sm.a[stage][r * (BK + 8) + kc], ok ? A + gm * lda + gk : A, ok);
            }
        }
        if constexpr (!TRANS) {
            for (int c = tid; c < BN * (BK / 8); c += kThreads) {
                const int r = c / (BK / 8), kc = (c % (BK / 8)) * 8;
                const int gn = n0 + r, gk = kb + kc;
                const bool ok = gn < N && gk < K;
                cp_async16(&sm.b[stage][r * (BK + 8) + kc], ok ? B + gn * ldb + gk : B, ok);
            }
        } else {
            // A: BK rows (k) x BM/8 chunks along M
            for (int c = tid; c < BK * (BM / 8); c += kThreads) {
                const int r = c / (BM / 8), mc = (c % (BM / 8)) * 8;
                const int gk = kb + r, gm = m0 + mc;
                const bool ok = gk < K && gm < M;
                cp_async16(&sm.a[stage][r * (BM + 8) + mc], ok ? A + gk * lda + gm : A, ok);
            }
            if constexpr (G == 2) {
                // B row r is the voxel p = kb + r, decomposed once for the thread's kCPT chunks
                const int r = (tid * kCPT) / (BN / 8);
                const int gk = kb + r;
                const bool kok = gk < K;
                const int v = kok ? gk : 0;
                const int t1 = fdiv(v, gx.fW), t2 = fdiv(t1, gx.fH), bb = fdiv(t2, gx.fD);
                const int x0 = v - t1 * gx.W, y0 = t1 - t2 * gx.H, z0 = t2 - bb * gx.D;
#pragma unroll
                for (int j = 0; j < kCPT; ++j) {
                    const int nc = ((tid * kCPT + j) % (BN / 8)) * 8;
                    const int xx = x0 + g_dx[j], yy = y0 + g_dy[j], zz = z0 + g_dz[j];
                    const bool ok = kok && g_nok[j] && zz >= 0 && zz < gx.D && yy >= 0 && yy < gx.H && xx >= 0 &&
                                    xx < gx.W;
                    const __nv_bfloat16 *src =
                        ok ? gx.x + ((((static_cast<int64_t>(bb) * gx.D + zz) * gx.H + yy) * gx.W + xx) * gx.C +
                                     g_ci[j])
                           : gx.x;
                    cp_async16(&sm.b[stage][r * (BN + 8) + nc], src, ok);
                }
            } else {
                for (int c = tid; c < BK * (BN / 8); c += kThreads) {
                    const int r = c / (BN / 8), nc = (c % (BN / 8)) * 8;
                    const int gk = kb + r, gn = n0 + nc;
                    const bool ok = gk < K && gn < N;
                    cp_async16(&sm.b[stage][r * (BN + 8) + nc], ok ? B + gk * ldb + gn : B, ok);
                }
            }
        }
        cp_async_commit();
    };

    float acc[MI][NI][4];
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < NI; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

    load_tile(0, ks0);
    for (int ks = ks0; ks < ks1; ++ks) {
        const int st = (ks - ks0) & 1;
        if (ks + 1 < ks1) {
            load_tile(st ^ 1, ks + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const __nv_bfloat16 *as = sm.a[st];
        const __nv_bfloat16 *bs = sm.b[st];
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[MI][4];
            uint32_t bf[NI][2];
            const int j = lane >> 3, r = lane & 7;
#pragma unroll
            for (int i = 0; i < MI; ++i) {
                const int mb = wm * TM + i * 16;
                if (!TRANS) {
                    const __nv_bfloat16 *p = as + (mb + r + 8 * (j & 1)) * (BK + 8) + kk + 8 * (j >> 1);
                    ldsm_x4(af[i][0], af[i][1], af[i][2], af[i][3], p);
                } else {
                    const __nv_bfloat16 *p = as + (kk + r + 8 * (j >> 1)) * (BM + 8) + mb + 8 * (j & 1);
                    ldsm_x4_t(af[i][0], af[i][1], af[i][2], af[i][3], p);
                }
            }
#pragma unroll
            for (int jn = 0; jn < NI; jn += 2) {
                const int nb = wn * TN + jn * 8;
                if (!TRANS) {
                    // matrices: (n 0-7, k 0-7), (n 0-7, k 8-15), (n 8-15, k 0-7), (n 8-15, k 8-15)
                    const __nv_bfloat16 *p = bs + (nb + r + 8 * (j >> 1)) * (BK + 8) + kk + 8 * (j & 1);
                    ldsm_x4(bf[jn][0], bf[jn][1], bf[jn + 1][0], bf[jn + 1][1], p);
                } else {
                    const __nv_bfloat16 *p = bs + (kk + r + 8 * (j & 1)) * (BN + 8) + nb + 8 * (j >> 1);
                    ldsm_x4_t(bf[jn][0], bf[jn][1], bf[jn + 1][0], bf[jn + 1][1], p);
                }
            }
#pragma unroll
            for (int i = 0; i < MI; ++i)
#pragma unroll
                for (int jn = 0; jn < NI; ++jn) mma_bf16(acc[i][jn], af[i], bf[jn][0], bf[jn][1]);
        }
        __syncthreads();
    }

    // epilogue: fragment (row = lane/4 [+8], col = 2*(lane%4) + {0,1})
    const int g = lane >> 2, tg = lane & 3;
    if constexpr (!TRANS) {
        if (part != nullptr) {
            // column sums of this tile's rows (and of their squares), for batch-norm
            // statistics: lanes, then the WM warps along M, in a fixed order;
            // part[blockIdx.x][0][col] and part[blockIdx.x][1][col]
            float (*red)[BN][2] = reinterpret_cast<float (*)[BN][2]>(&sm);
#pragma unroll
            for (int jn = 0; jn < NI; ++jn)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    float cs = 0.0f, cq = 0.0f;
#pragma unroll
                    for (int i = 0; i < MI; ++i)
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int row = m0 + wm * TM + i * 16 + g + 8 * h;
                            const float v = row < M ? acc[i][jn][2 * h + e] : 0.0f;
                            cs += v;
                            cq += v * v;
                        }
#pragma unroll
                    for (int o = 4; o < 32; o <<= 1) {
                        cs += __shfl_xor_sync(0xffffffffu, cs, o);
                        cq += __shfl_xor_sync(0xffffffffu, cq, o);
                    }
                    if (g == 0) {
                        const int col = wn * TN + jn * 8 + 2 * tg + e;
                        red[wm][col][0] = cs;
                        red[wm][col][1] = cq;
                    }
                }
            __syncthreads();
            for (int col = tid; col < BN; col += kThreads) {
                float cs = 0.0f, cq = 0.0f;
                for (int w = 0; w < WM; ++w) {
                    cs += red[w][col][0];
                    cq += red[w][col][1];
                }
                if (n0 + col < N) {
                    part[(static_cast<int64_t>(blockIdx.x) * 2) * N + n0 + col] = cs;
                    part[(static_cast<int64_t>(blockIdx.x) * 2 + 1) * N + n0 + col] = cq;
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int jn = 0; jn < NI; ++jn)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m0 + wm * TM + i * 16 + g + 8 * h;
                const int col = n0 + wn * TN + jn * 8 + 2 * tg;
                if (row >= M) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (col + e >= N) continue;
                    float *dst = C + row * ldc + col + e;
                    if (TRANS) {
                        // split-K: with part set, each split writes its own slice part[blockIdx.z][M][N]
                        // (summed afterwards in split order); otherwise atomically into C
                        if (part != nullptr)
                            part[(static_cast<int64_t>(blockIdx.z) * M + row) * N + col + e] = acc[i][jn][2 * h + e];
                        else
                            atomicAdd(dst, acc[i][jn][2 * h + e]);
                    } else {
                        *dst = acc[i][jn][2 * h + e];
                    }
                }
            }
}

}  // namespace gemm
}  // namespace nsfrb
