// 3x3x3 convolution with zero padding 1 of a channels-last volume x[b][z][y][x][CI] with
// weights w[CO][27][CI] (tap = (dz * 3 + dy) * 3 + dx), FP32 output y[voxel][CO], on the
// 5th-generation tensor cores: tcgen05.mma (kind::f16, BF16 operands in shared memory, FP32
// accumulator in tensor memory).
//
// The GEMM view is D[voxel][co] = sum over (tap, ci) of x[voxel + tap][ci] w[co][tap][ci].  A CTA
// keeps all the weights in shared memory and walks output bricks of 1 x 16 x 8 voxels (z, y, x):
// M = 128 rows, row m = 8 y + x.  Each brick's 3 x 18 x 10 input halo is stored per 8-channel
// chunk as [z][y][x][8 channels], which is the canonical K-major layout without swizzle: a core
// matrix is 8 consecutive x (16 bytes each), successive y rows are 10 x 16 bytes apart (the
// stride between 8-row groups) and channel chunks are one halo plane apart (the stride between
// K core matrices).  A tap is then only a start-address offset of the A descriptor, so one
// brick is 27 x CI / 16 MMAs of 128 x CO x 16 with no data movement between taps.  The weights
// are stored [tap][chunk][co][8] (the same layout for B).
//
// Warp roles, one CTA of 8 warps, synchronised only through mbarriers (bounded waits):
//  * warp 0 allocates tensor memory; its lane 0 issues the MMAs of a brick once its halo is in
//    shared memory and its accumulator (one of two, CO columns each) has been drained, and
//    commits them to "halo free" and "accumulator full" barriers;
//  * warps 1-3 copy halos (16-byte cp.async from offsets precomputed per thread, zero outside
//    the volume) into a ring of NS buffers with up to NS - 1 bricks in flight, and mark a
//    buffer full once their copies have landed (after a proxy fence: the tensor cores read
//    through the async proxy);
//  * warps 4-7 (TMEM lanes 0-127) read an accumulator out, mark it empty, reduce the column
//    sums of y and y^2 for batch norm in a fixed order, and write y (FP32) through a
//    shared-memory tile so that each warp stores contiguous 512-byte runs.
// Measured on the 16 -> 32 channel layer (B = 64, 32^3): the per-tap index and descriptor
// arithmetic of a rolled tap loop cost ~180 cycles per MMA, row-per-thread stores of y cost
// ~1000 L1 wavefronts per brick, and a TMA box with 16-byte rows (one channel chunk of one
// voxel) moved the halos several times slower than the copies; hence the unrolled taps, the
// staged stores and the copies.  One CTA issuing 128 x 32 x 16 MMAs reaches ~67 cycles per
// MMA, two CTAs per SM ~40 (the shared-memory operand read of 5 KB per MMA): N = 32 caps the
// tensor pipe at about 40 % of its BF16 peak.
// On a timeout the kernel latches an error bit, every role stops, the MMA warp waits
// (bounded) for its MMAs in flight and tensor memory is freed.  `stall` (tests only) keeps the
// producers from ever marking a halo full, so that this path runs on demand.
#pragma once

#include <cuda_bf16.h>

#include "async_copy.cuh"
#include "gemm.cuh"

namespace nsfrb {
namespace conv3tc {

using bf16 = __nv_bfloat16;

constexpr int BY = 16, BX = 8;                                     // output brick (one z plane)
constexpr int HZ = 3, HY = BY + 2, HX = BX + 2, HV = HZ * HY * HX;   // its halo: 540 voxels
constexpr int kThreads = 256;                                      // 8 warps (roles above)
constexpr int kProducers = 96;                                     // warps 1-3
constexpr uint32_t kPlane = 8704;   // bytes per channel chunk of a halo (540 x 16, padded to 128)
constexpr int kErrWait = 4;         // error bit: a tensor-core wait timed out

constexpr size_t kSmemMax = 227 * 1024;   // opt-in shared memory per CTA

template <int CI, int CO, int NS_>
struct Layout {
    static constexpr int KC = CI / 8;                               // 16-byte channel chunks
    static constexpr size_t h_bytes = static_cast<size_t>(KC) * kPlane;    // one halo buffer
    static constexpr size_t w_bytes = static_cast<size_t>(27) * KC * CO * 16;
    static constexpr size_t red_bytes = sizeof(float) * 2 * 4 * CO * 2;   // [2][4 warps][CO][2]
    static constexpr size_t stg_bytes = sizeof(float) * 128 * (CO + 4);   // output tile [128][CO + 4]
    static constexpr size_t off_w = NS_ * h_bytes;
    static constexpr size_t off_stg = off_w + w_bytes;
    static constexpr size_t off_red = off_stg + stg_bytes;
    static constexpr size_t off_bar = off_red + red_bytes;          // 2 NS + 4 mbarriers, TMEM slot, flag
    static constexpr size_t smem = off_bar + (2 * NS_ + 4) * 8 + 16;
};

template <int CI, int CO>
struct Shape {
    static_assert(CI % 16 == 0 && CO % 16 == 0 && CO <= 64, "CI multiple of 16, CO in {16, 32, 48, 64}");
    // three halo buffers (two bricks in flight) when they fit, else two
    static constexpr int NS = (Layout<CI, CO, 3>::smem <= kSmemMax) ? 3 : 2;
    using L = Layout<CI, CO, NS>;
    static constexpr int KC = L::KC;
    static constexpr size_t h_bytes = L::h_bytes, w_bytes = L::w_bytes;
    static constexpr size_t off_w = L::off_w, off_stg = L::off_stg, off_red = L::off_red, off_bar = L::off_bar;
    static constexpr size_t smem = L::smem;
    static constexpr int kPer = (HV * KC + kProducers - 1) / kProducers;   // halo chunks per producer
    static constexpr uint32_t cols = (2 * CO <= 32) ? 32u : (2 * CO <= 64 ? 64u : 128u);   // power of 2
    // instruction descriptor (kind::f16): D FP32, A and B BF16, both K-major, N = CO, M = 128
    static constexpr uint32_t idesc =
        (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(CO >> 3) << 17) | (static_cast<uint32_t>(128 >> 4) << 24);
};

// Shared-memory matrix descriptor, no swizzle: start address, the byte offset between core
// matrices along K (lbo) and along M or N (sbo), all in 16-byte units; bit 46 is the fixed
// descriptor version of sm_100.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((addr >> 4) & 0x3FFFu) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     dev::smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Column sums over the warp's 32 lanes of N = 16 or 32 values per lane, by halving exchanges
// in a fixed order: afterwards v[0] of lane l is the sum of column l mod N.
template <int N>
__device__ __forceinline__ float lane_col_sum(float (&v)[N], int lane) {
#pragma unroll
    for (int h = N / 2; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const float send = up ? v[j] : v[j + h];
            const float keep = up ? v[j + h] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    if constexpr (N == 16) v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16);
    return v[0];
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(dev::smem_u32(bar)) : "memory");
}

// Bricks are numbered b-major, then z, y, x: brick (b, z, yb, xb) covers the plane z,
// y in [16 yb, 16 yb + 16), x in [8 xb, 8 xb + 8).  H % 16 = W % 8 = 0.
template <int CI, int CO>
__global__ void __launch_bounds__(kThreads, 1) conv3_tc_kernel(const bf16 *__restrict__ x, const bf16 *__restrict__ w,
                                                            float *__restrict__ y, float *__restrict__ part, int D,
                                                            int H, int W, int n_bricks, int *__restrict__ err,
                                                            int stall) {
    using S = Shape<CI, CO>;
    constexpr int KC = S::KC;
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int NS = S::NS;
    unsigned char *s_h = smem;                      // [NS][KC][kPlane]
    unsigned char *s_w = smem + S::off_w;           // [27][KC][CO][16 B]
    float *s_stg = reinterpret_cast<float *>(smem + S::off_stg);   // [128][CO + 4]
    float (*red)[4][CO][2] = reinterpret_cast<float (*)[4][CO][2]>(smem + S::off_red);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + S::off_bar);
    unsigned long long *hfull = bars, *hfree = bars + NS, *afull = bars + 2 * NS, *afree = bars + 2 * NS + 2;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + 2 * NS + 4);
    int *s_fail = reinterpret_cast<int *>(s_tmem + 1);
    volatile int *fail = s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nxb = W / BX, nyb = H / BY;
    const int G = gridDim.x;
    const int bi0 = blockIdx.x;
    const int n_mine = (bi0 < n_bricks) ? (n_bricks - 1 - bi0) / G + 1 : 0;   // this CTA's bricks

    auto origin = [&](int bi, int &b, int &z0, int &y0, int &x0) {
        const int xb = bi % nxb, t1 = bi / nxb, yb = t1 % nyb, t2 = t1 / nyb;
        z0 = t2 % D;
        b = t2 / D;
        y0 = yb * BY;
        x0 = xb * BX;
    };
    // a bounded wait that also gives up once another role has failed
    auto wait = [&](unsigned long long *bar, uint32_t parity) -> bool {
        if (dev::mbar_try_wait(bar, parity)) return true;
        const unsigned long long t0 = dev::global_ns();
        while (!dev::mbar_try_wait(bar, parity)) {
            if (*fail) return false;
            if (dev::global_ns() - t0 > dev::kWaitNs) {
                *fail = 1;
                return false;
            }
            __nanosleep(64);
        }
        return true;
    };

    // ---- setup: barriers, tensor memory, weights (re-laid out as [tap][chunk][co][8])
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            dev::mbar_init(&hfull[i], kProducers);
            dev::mbar_init(&hfree[i], 1);
        }
        dev::mbar_init(&afull[0], 1);
        dev::mbar_init(&afull[1], 1);
        dev::mbar_init(&afree[0], 128);
        dev::mbar_init(&afree[1], 128);
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dev::smem_u32(s_tmem)),
                     "r"(S::cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int c = tid; c < CO * 27 * KC; c += kThreads) {
        const int co = c / (27 * KC), r = c - co * (27 * KC);   // r = tap * KC + chunk
        gemm::cp_async16(s_w + (static_cast<size_t>(r) * CO + co) * 16, w + static_cast<int64_t>(co) * 27 * CI + r * 8,
                         true);
    }
    gemm::cp_async_commit();
    gemm::cp_async_wait<0>();
    dev::fence_proxy_async();   // the weights are read by the tensor cores (async proxy)
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp == 0) {
        // ---------------- MMA issuer
        int last = -1;   // the last brick whose MMAs were committed
        if (lane == 0) {
            const uint32_t b0 = dev::smem_u32(s_w);
            const uint64_t bd0 = sdesc(b0, CO * 16, 128);
            for (int j = 0; j < n_mine; ++j) {
                const int s = j & 1, hs = j % NS;
                if (!wait(&hfull[hs], (j / NS) & 1)) break;                    // halo j in buffer hs
                if (j >= 2 && !wait(&afree[s], ((j >> 1) - 1) & 1)) break;      // accumulator s drained
                tc_fence_after();
                const uint64_t ad0 = sdesc(dev::smem_u32(s_h + static_cast<size_t>(hs) * KC * kPlane), kPlane, HX * 16);
                const uint32_t d = tmem + static_cast<uint32_t>(s * CO);
                // every descriptor is the base one plus a compile-time start-address offset (16-byte units)
#pragma unroll
                for (int tap = 0; tap < 27; ++tap) {
                    const uint32_t a_off = static_cast<uint32_t>(((tap / 9) * HY + (tap / 3) % 3) * HX + tap % 3);
#pragma unroll
                    for (int ks = 0; ks < CI / 16; ++ks) {
                        const uint64_t ad = ad0 + a_off + static_cast<uint32_t>(2 * ks) * (kPlane >> 4);
                        const uint64_t bd = bd0 + static_cast<uint32_t>((tap * KC + 2 * ks) * CO);
                        umma_f16(d, ad, bd, S::idesc, (tap | ks) != 0);
                    }
                }
                umma_commit(&hfree[hs]);   // the halo buffer is free once these MMAs have read it
                umma_commit(&afull[s]);   // ... and the accumulator is complete
                last = j;
            }
            // after a failure: the MMAs in flight complete before tensor memory is freed
            if (*fail && last >= 0) dev::mbar_wait(&afull[last & 1], (last >> 1) & 1);
        }
        __syncwarp();
    } else if (warp < 4) {
        // ---------------- halo producers: chunk k of this thread is halo voxel / channel chunk
        // c = t + 96 k; its shared-memory offset and its element offset from the halo's corner
        // voxel are the same for every brick
        const int t = tid - 32;
        int soff[S::kPer], goff[S::kPer], cz[S::kPer];   // cz: packed (hz, hy, hx), -1 past the end
#pragma unroll
        for (int k = 0; k < S::kPer; ++k) {
            const int c = t + kProducers * k;
            if (c < HV * KC) {
                const int hv = c / KC, kc = c - hv * KC;
                const int hz = hv / (HY * HX), hy = (hv / HX) % HY, hx = hv % HX;
                soff[k] = kc * static_cast<int>(kPlane) + hv * 16;
                goff[k] = ((hz * H + hy) * W + hx) * CI + kc * 8;
                cz[k] = (hz << 16) | (hy << 8) | hx;
            } else {
                soff[k] = goff[k] = 0;
                cz[k] = -1;
            }
        }
        auto issue = [&](int j) {
            int b, z0, y0, x0;
            origin(bi0 + j * G, b, z0, y0, x0);
            const bf16 *corner = x + (((static_cast<int64_t>(b) * D + z0 - 1) * H + y0 - 1) * W + x0 - 1) * CI;
            unsigned char *dst = s_h + static_cast<size_t>(j % NS) * KC * kPlane;
#pragma unroll
            for (int k = 0; k < S::kPer; ++k) {
                if (cz[k] < 0) continue;
                const int zz = z0 - 1 + (cz[k] >> 16), yy = y0 - 1 + ((cz[k] >> 8) & 255), xx = x0 - 1 + (cz[k] & 255);
                const bool ok = zz >= 0 && zz < D && yy >= 0 && yy < H && xx >= 0 && xx < W;
                gemm::cp_async16(dst + soff[k], ok ? corner + goff[k] : x, ok);
            }
            gemm::cp_async_commit();
        };
        // up to NS - 1 halos in flight: after issuing brick j, brick j - (NS - 2) is awaited; a
        // buffer is refilled once the MMAs that read it are done
        int arrived = 0;   // bricks marked full
        for (int j = 0; j < n_mine; ++j) {
            if (j >= NS && !wait(&hfree[j % NS], ((j / NS) - 1) & 1)) break;
            issue(j);
            if (j >= NS - 2) {
                gemm::cp_async_wait<NS - 2>();   // brick `arrived` (this thread's part) has landed
                dev::fence_proxy_async();
                if (!stall) mbar_arrive(&hfull[arrived % NS]);
                ++arrived;
            }
        }
        gemm::cp_async_wait<0>();
        if (!*fail && !stall) {
            dev::fence_proxy_async();
            for (; arrived < n_mine; ++arrived) mbar_arrive(&hfull[arrived % NS]);
        }
    } else {
        // ---------------- epilogue: accumulator row m = TMEM lane 32 (warp - 4) + lane
        const int q = warp - 4, m = 32 * q + lane;
        for (int j = 0; j < n_mine; ++j) {
            const int s = j & 1;
            if (!wait(&afull[s], (j >> 1) & 1)) break;
            tc_fence_after();
            const int bi = bi0 + j * G;
            int b, z0, y0, x0;
            origin(bi, b, z0, y0, x0);
            const uint32_t trow = tmem + (static_cast<uint32_t>(32 * q) << 16) + static_cast<uint32_t>(s * CO);
#pragma unroll
            for (int c0 = 0; c0 < CO; c0 += 16) {
                float v[16];
                tmem_ld16(trow + c0, v);
                tmem_wait_ld();
                float4 *st = reinterpret_cast<float4 *>(s_stg + m * (CO + 4) + c0);
#pragma unroll
                for (int e = 0; e < 4; ++e) st[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
                if (part != nullptr) {
                    float sq[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) sq[e] = v[e] * v[e];
                    const float cs = lane_col_sum<16>(v, lane);
                    const float cq = lane_col_sum<16>(sq, lane);
                    if (lane < 16) {
                        red[s][q][c0 + lane][0] = cs;
                        red[s][q][c0 + lane][1] = cq;
                    }
                }
            }
            // the accumulator has been read: the MMAs of brick j + 2 may overwrite it
            tc_fence_before();
            mbar_arrive(&afree[s]);
            asm volatile("bar.sync 1, 128;" ::: "memory");   // the four epilogue warps: tile and sums staged
            {
                // brick row r = 8 y + x is voxel (z0, y0 + y, x0 + x): 8 voxels x CO floats are contiguous
                const int64_t pb = ((static_cast<int64_t>(b) * D + z0) * H + y0) * W + x0;
#pragma unroll
                for (int i = 0; i < CO / 4; ++i) {
                    const int f = m + 128 * i, r = f / (CO / 4), c4 = f - r * (CO / 4);
                    *reinterpret_cast<float4 *>(y + (pb + (r >> 3) * W + (r & 7)) * CO + 4 * c4) =
                        *reinterpret_cast<const float4 *>(s_stg + r * (CO + 4) + 4 * c4);
                }
            }
            if (part != nullptr) {
                for (int col = m; col < CO; col += 128) {
                    float cs = 0.0f, cq = 0.0f;
                    for (int r = 0; r < 4; ++r) {
                        cs += red[s][r][col][0];
                        cq += red[s][r][col][1];
                    }
                    part[(static_cast<int64_t>(bi) * 2) * CO + col] = cs;
                    part[(static_cast<int64_t>(bi) * 2 + 1) * CO + col] = cq;
                }
            }
            asm volatile("bar.sync 1, 128;" ::: "memory");   // the tile is read before the next brick's
        }
    }

    // ---- all roles done: report, free tensor memory
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *fail) atomicOr(err, kErrWait);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::cols) : "memory");
    }
}

}  // namespace conv3tc
}  // namespace nsfrb
