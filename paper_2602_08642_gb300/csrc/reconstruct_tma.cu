// TMA-pipelined reconstruction of one pyramid level (Appendix A of
// arXiv 2602.08642; tone map of Sec. 5 as the full-resolution epilogue).
//
// Persistent kernel, one 512-thread CTA per SM (two threads per pixel), each
// CTA walking the 64 x 4 pixel tiles t = blockIdx.x, blockIdx.x + gridDim.x,
// ...  (64 x 4 rather than 32 x 8: each logit plane arrives as 256-byte rows,
// which measured 8 % faster at full resolution).  For every tile one thread
// issues up to four bulk tensor copies (cp.async.bulk.tensor) into a stage
// of shared memory, all completing on the stage's mbarrier:
//   logits  box 64 x 4 x C       (C = 25, 29 or 54 planes)
//   noisy   box 72 x 8 x 3       (the tile plus a 2-pixel halo; x starts at
//                                 x0 - 4 so that it is 16-byte aligned)
//   warped  box 72 x 8 x 3       (full resolution only: W_t L_{t-1}, written
//                                 by warp_prev_kernel, on the same halo)
//   coarse  box 40 x 3 x 3       (below a coarser level: the cells of L-hat of
//                                 that level the tile's upsampling taps read;
//                                 x starts at x0 / 2 - 4, 16-byte aligned)
// NS stages are in flight, so HBM keeps streaming while the threads compute.
// There is no CTA-wide barrier in the tile loop: each warp waits on the
// stage's mbarrier, the last warp done with a stage refills it, and the two
// warps of a pixel row meet on their own mbarrier.
// Halo cells outside the image arrive zero-filled and are never read: tiles
// whose 5 x 5 footprint crosses the border index their clamp-to-edge source
// cells.  The disocclusion mask is a plain load issued one tile ahead.
// Every mbarrier wait is bounded in time (kWaitNs of %globaltimer): on expiry
// the CTA records SPP_ERR_TIMEOUT, waits (bounded the same way) for the
// copies it has issued and exits.  Those copies read in-bounds boxes of this
// kernel's own inputs and complete without help from any other CTA, so the
// drain wait runs out only if the memory system itself has failed.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "recon_common.cuh"
#include "tma_host.cuh"

namespace spp {
namespace {

constexpr int kPX = 64;            // tile width (a multiple of 32)
constexpr int kPY = 256 / kPX;     // tile height
constexpr int kPixels = kPX * kPY;  // 256 pixels per tile
constexpr int kWarpsPerRow = kPX / 32;
static_assert(kPX % 32 == 0 && kPixels == 256, "tile of 256 pixels, whole warps per row");
constexpr int kThreads = 2 * kPixels; // two threads per pixel, each summing half of the taps
constexpr int kBoxX = kPX + 8;     // noisy / warped box width, x from x0 - 4
constexpr int kBoxY = kPY + 4;     // rows y0 - 2 .. y0 + kPY + 1
constexpr int kCoarseX = kPX / 2 + 8;  // coarse columns x0/2 - 4 .. x0/2 + kPX/2 + 3
constexpr int kCoarseY = kPY / 2 + 1;  // coarse rows y0/2 .. y0/2 + kPY/2
constexpr unsigned long long kWaitNs = 100000000ull;  // 100 ms per wait

template <int C, bool UP, bool TEMP>
struct Stage {
    static constexpr int kLogitFloats = kPX * kPY * C;
    static constexpr int kNoisyFloats = kBoxX * kBoxY * 3;
    static constexpr int kWarpedFloats = TEMP ? kBoxX * kBoxY * 3 : 0;
    static constexpr int kCoarseFloats = UP ? kCoarseX * kCoarseY * 3 : 0;
    static constexpr int kCoarseSlot = (kCoarseFloats + 31) / 32 * 32;  // 128-byte multiple
    // stage stride in floats, and the bytes its copies bring
    static constexpr int kFloats = kLogitFloats + kNoisyFloats + kWarpedFloats + kCoarseSlot;
    static constexpr uint32_t kBytes =
        (kLogitFloats + kNoisyFloats + kWarpedFloats + kCoarseFloats) * 4u;
    static_assert((kLogitFloats * 4) % 128 == 0 && (kNoisyFloats * 4) % 128 == 0 &&
                      (kFloats * 4) % 128 == 0,
                  "box alignment");
};

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// The suspend-time hint lets a waiting thread sleep in the barrier instead
// of re-polling (each call still returns, so the caller's bound holds).
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Gives up (returns false) once kWaitNs have passed since the first poll.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(float *dst, const CUtensorMap *map, uint64_t *bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// ------------------------------------------------------------ the kernel
struct TileGeom {
    int tiles_x, num_tiles;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int C, bool UP, bool TEMP, bool TONE, int NS>
__global__ void __launch_bounds__(kThreads, 1)
recon_tma_kernel(const __grid_constant__ CUtensorMap map_logits,
                 const __grid_constant__ CUtensorMap map_noisy,
                 const __grid_constant__ CUtensorMap map_warped,
                 const __grid_constant__ CUtensorMap map_coarse, const uint8_t *__restrict__ mask,
                 int Wl, int Hl, TileGeom geom,
                 float *__restrict__ out, float *__restrict__ out_ldr, ToneArgs tm,
                 int32_t *status, int stall_tile) {
    using S = Stage<C, UP, TEMP>;
    static_assert(!TEMP || UP, "temporal term only at full resolution below a coarser level");
    static_assert(NS <= 8, "stage bookkeeping holds 8 stages");
    constexpr int kWarps = kThreads / 32;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // offset arithmetic on the shared array keeps the accesses in the shared
    // window (plain shared loads rather than generic ones)
    unsigned char *base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    uint64_t *full = reinterpret_cast<uint64_t *>(base);            // [NS]   at +0
    uint64_t *pair = reinterpret_cast<uint64_t *>(base + 64);       // [8]    at +64
    int *done = reinterpret_cast<int *>(base + 128);                // [NS]   at +128
    int *uses = reinterpret_cast<int *>(base + 160);                // [NS]   at +160
    float *stages = reinterpret_cast<float *>(base + 256);
    float *part = stages + NS * S::kFloats;  // [2][5][256] partials, half 1 -> half 0

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long Nl = static_cast<long long>(Wl) * Hl;
    const int G = gridDim.x;
    const int my_tiles =
        blockIdx.x < geom.num_tiles ? (geom.num_tiles - 1 - blockIdx.x) / G + 1 : 0;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            done[s] = 0;
            uses[s] = 0;
        }
        for (int r = 0; r < 8; ++r) mbar_init(&pair[r], 64);
        fence_mbar_init();
    }
    __syncthreads();
    pdl_wait();  // the previous kernel's outputs (this level's inputs) are complete
    pdl_trigger();
    if (my_tiles == 0) return;

    auto tile_xy = [&](int k, int &x0, int &y0) {
        const int t = blockIdx.x + k * G;
        x0 = (t % geom.tiles_x) * kPX;
        y0 = (t / geom.tiles_x) * kPY;
    };
    auto logits_of = [&](int s) { return stages + s * S::kFloats; };
    auto noisy_of = [&](int s) { return stages + s * S::kFloats + S::kLogitFloats; };
    auto warped_of = [&](int s) { return stages + s * S::kFloats + S::kLogitFloats + S::kNoisyFloats; };
    auto coarse_of = [&](int s) {
        return stages + s * S::kFloats + S::kLogitFloats + S::kNoisyFloats + S::kWarpedFloats;
    };

    auto issue = [&](int k) {
        const int s = k % NS;
        int x0, y0;
        tile_xy(k, x0, y0);
        // test of the bounded waits: this tile's stage is never filled (and
        // keeps its previous use, whose copies have all landed)
        if (blockIdx.x + k * G == stall_tile) return;
        uses[s] = k / NS + 1;
        fence_proxy_async();
        mbar_expect_tx(&full[s], S::kBytes);
        tma_load_3d(logits_of(s), &map_logits, &full[s], x0, y0, 0);
        tma_load_3d(noisy_of(s), &map_noisy, &full[s], x0 - 4, y0 - 2, 0);
        if (TEMP) tma_load_3d(warped_of(s), &map_warped, &full[s], x0 - 4, y0 - 2, 0);
        if (UP) tma_load_3d(coarse_of(s), &map_coarse, &full[s], x0 / 2 - 4, y0 / 2, 0);
    };
    if (tid == 0)
        for (int k = 0; k < NS && k < my_tiles; ++k) issue(k);
    __syncthreads();

    // After a wait gave up: record it, wait (bounded) for the copies this CTA
    // issued on every stage, and let the caller return.  Every wait in this
    // kernel is bounded, so the other warps reach the same point.
    auto abort = [&]() {
        set_status(status, SPP_ERR_TIMEOUT);
        if (lane == 0)
            for (int s = 0; s < NS; ++s) {
                const int u = *reinterpret_cast<volatile int *>(&uses[s]);
                if (u > 0) (void)mbar_wait_bounded(&full[s], static_cast<uint32_t>((u - 1) & 1));
            }
    };
    // This warp has finished reading tile k's stage; the last of the 16 warps
    // to get here refills the stage with tile k + NS.
    auto release = [&](int k) {
        __syncwarp();
        if (lane == 0) {
            const int s = k % NS;
            __threadfence_block();  // this warp's reads of the stage come first
            if (atomicAdd(&done[s], 1) == kWarps - 1) {
                __threadfence_block();
                done[s] = 0;
                if (k + NS < my_tiles) issue(k + NS);
            }
        }
        __syncwarp();
    };

    // The two threads of a pixel: half 0 (warps 0-7) and half 1 (warps 8-15)
    // sum disjoint parts of the joint softmax; half 1 hands its (max, weight
    // sum, weighted sums) to half 0, which merges, normalises, tone-maps and
    // stores.  Warp w and warp w + 8 hold the same 32 pixels of a tile row
    // and meet on pair[w].
    //   temporal level: half 0 = kappa_d taps; half 1 = kappa_u + kappa_t taps
    //   other levels:   half 0 = kappa_d rows 0-2; half 1 = rows 3-4 + kappa_u
    const int half = warp >> 3;
    const int wr = warp & 7;
    const int ty = wr / kWarpsPerRow, tx = (wr % kWarpsPerRow) * 32 + lane;
    const int p = ty * kPX + tx;

    // the disocclusion mask, loaded one tile ahead (half 1)
    bool use_t = false;
    auto prefetch = [&](int k, bool &ut) {
        int x0, y0;
        tile_xy(k, x0, y0);
        const int xc = min(x0 + tx, Wl - 1), yc = min(y0 + ty, Hl - 1);
        ut = !(mask && __ldg(mask + static_cast<long long>(yc) * Wl + xc));
    };
    if (TEMP && half == 1) prefetch(0, use_t);
    // the upsampling term: kappa_u weights on the coarse cells of the stage
    constexpr int kCP = kCoarseX * kCoarseY;
    auto up_taps = [&](int s, int x0, int y0, const float *lu, float mL, float &ws, float &b0,
                       float &b1, float &b2) {
        const float *cb = coarse_of(s);
        const int xc = min(x0 + tx, Wl - 1), yc = min(y0 + ty, Hl - 1);
        const int Wc = Wl >> 1, Hc = Hl >> 1;
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int cx = min((xc + i) >> 1, Wc - 1) - (x0 / 2 - 4);
                const int cy = min((yc + j) >> 1, Hc - 1) - y0 / 2;
                const int o = cy * kCoarseX + cx;
                const float e = ex2_approx(fmaf(lu[2 * j + i], kLog2e, -mL));
                ws += e;
                b0 = fmaf(e, cb[o], b0);
                b1 = fmaf(e, cb[kCP + o], b1);
                b2 = fmaf(e, cb[2 * kCP + o], b2);
            }
    };

    constexpr int kNC = kBoxX * kBoxY;
    constexpr int kPlane = kPX * kPY;
    for (int k = 0; k < my_tiles; ++k) {
        const int s = k % NS;
        int x0, y0;
        tile_xy(k, x0, y0);
        if (!mbar_wait_bounded(&full[s], static_cast<uint32_t>((k / NS) & 1))) {
            abort();
            return;
        }
        bool use_tn = false;
        if (TEMP && half == 1 && k + 1 < my_tiles) prefetch(k + 1, use_tn);

        // tiles whose 5 x 5 footprint crosses the image border read clamped
        // cells (the zero-filled ones are never read)
        const bool edge = (x0 - 2 < 0) || (x0 + kPX + 1 > Wl - 1) || (y0 - 2 < 0) ||
                          (y0 + kPY + 1 > Hl - 1);
        // this thread's part of the joint softmax, from shared memory
        const float *lgs = logits_of(s) + p;
        const float *nz = noisy_of(s);
        float m, wsum = 0.0f, a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
        auto gather_rows = [&](const float *img, const float *lgv, int jr0, int jr1, float mL) {
            if (!edge) {  // CTA-uniform: constant offsets from the pixel's cell
                const float *b = img + ty * kBoxX + tx + 2;
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    if (j < jr0 || j >= jr1) continue;
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        const float e = ex2_approx(fmaf(lgv[(j - jr0) * 5 + i], kLog2e, -mL));
                        const int o = j * kBoxX + i;
                        wsum += e;
                        a0 = fmaf(e, b[o], a0);
                        a1 = fmaf(e, b[kNC + o], a1);
                        a2 = fmaf(e, b[2 * kNC + o], a2);
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < 5; ++j) {
                    if (j < jr0 || j >= jr1) continue;
                    const int rb = (clampi(y0 + ty + j - 2, 0, Hl - 1) - (y0 - 2)) * kBoxX;
#pragma unroll
                    for (int i = 0; i < 5; ++i) {
                        const float e = ex2_approx(fmaf(lgv[(j - jr0) * 5 + i], kLog2e, -mL));
                        const int o = rb + clampi(x0 + tx + i - 2, 0, Wl - 1) - (x0 - 4);
                        wsum += e;
                        a0 = fmaf(e, img[o], a0);
                        a1 = fmaf(e, img[kNC + o], a1);
                        a2 = fmaf(e, img[2 * kNC + o], a2);
                    }
                }
            }
        };
        if (TEMP) {
            if (half == 0) {
                float lg[25];
#pragma unroll
                for (int kk = 0; kk < 25; ++kk) lg[kk] = lgs[kk * kPlane];
                m = lg[0];
#pragma unroll
                for (int kk = 1; kk < 25; ++kk) m = fmaxf(m, lg[kk]);
                gather_rows(nz, lg, 0, 5, m * kLog2e);
            } else {
                float lg[29];
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) lg[kk] = lgs[(25 + kk) * kPlane];
                m = fmaxf(fmaxf(lg[0], lg[1]), fmaxf(lg[2], lg[3]));
                if (use_t) {
#pragma unroll
                    for (int kk = 0; kk < 25; ++kk) lg[4 + kk] = lgs[(29 + kk) * kPlane];
#pragma unroll
                    for (int kk = 4; kk < 29; ++kk) m = fmaxf(m, lg[kk]);
                }
                const float mL = m * kLog2e;
                up_taps(s, x0, y0, lg, mL, wsum, a0, a1, a2);
                if (use_t) gather_rows(warped_of(s), lg + 4, 0, 5, mL);
            }
        } else {
            const int jr0 = half == 0 ? 0 : 3, jr1 = half == 0 ? 3 : 5;
            float lg[15];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int i = 0; i < 5; ++i)
                    lg[r * 5 + i] = (jr0 + r < jr1) ? lgs[((jr0 + r) * 5 + i) * kPlane] : -INFINITY;
            float lu[4];
            m = lg[0];
#pragma unroll
            for (int kk = 1; kk < 15; ++kk) m = fmaxf(m, lg[kk]);
            if (UP && half == 1) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    lu[q] = lgs[(25 + q) * kPlane];
                    m = fmaxf(m, lu[q]);
                }
            }
            const float mL = m * kLog2e;
            if (half == 0)
                gather_rows(nz, lg, 0, 3, mL);
            else
                gather_rows(nz, lg, 3, 5, mL);
            if (UP && half == 1) up_taps(s, x0, y0, lu, mL, wsum, a0, a1, a2);
        }
        release(k);

        float *pk = part + (k & 1) * 5 * kPixels;
        if (half == 1) {
            pk[0 * kPixels + p] = m;
            pk[1 * kPixels + p] = wsum;
            pk[2 * kPixels + p] = a0;
            pk[3 * kPixels + p] = a1;
            pk[4 * kPixels + p] = a2;
            use_t = use_tn;
        }
        // rendezvous of the pixel row's two warps (bounded)
        mbar_arrive(&pair[wr]);
        if (!mbar_wait_bounded(&pair[wr], static_cast<uint32_t>(k & 1))) {
            abort();
            return;
        }
        const int x = x0 + tx, y = y0 + ty;
        if (half == 0 && x < Wl && y < Hl) {
            const float m1 = pk[p], w1 = pk[kPixels + p];
            const float M = fmaxf(m, m1);
            const float s0 = ex2_approx((m - M) * kLog2e), s1 = ex2_approx((m1 - M) * kLog2e);
            const float inv = rcp_approx(wsum * s0 + w1 * s1);
            const float o0 = (a0 * s0 + pk[2 * kPixels + p] * s1) * inv;
            const float o1 = (a1 * s0 + pk[3 * kPixels + p] * s1) * inv;
            const float o2 = (a2 * s0 + pk[4 * kPixels + p] * s1) * inv;
            const long long op = static_cast<long long>(y) * Wl + x;
            __stcs(out + op, o0);
            __stcs(out + Nl + op, o1);
            __stcs(out + 2 * Nl + op, o2);
            if (TONE) {
                float r, g, b;
                tone_map(o0, o1, o2, tm, r, g, b);
                __stcs(out_ldr + op, r);
                __stcs(out_ldr + Nl + op, g);
                __stcs(out_ldr + 2 * Nl + op, b);
            }
        }
    }
}

// W_t L_{t-1}: bilinear sample of the previous HDR output at (x + mv_x,
// y + mv_y), pixel centres at integers, the position clamped to the frame.
// The fraction is taken from the motion vector itself so that it is exact.
__global__ void __launch_bounds__(256)
warp_prev_kernel(const float *__restrict__ prev, const float *__restrict__ mv, int Wl, int Hl,
                 float *__restrict__ warped) {
    const int gx = blockIdx.x * 64 + (threadIdx.x & 63);
    const int gy = blockIdx.y * 4 + (threadIdx.x >> 6);
    if (gx >= Wl || gy >= Hl) return;
    const long long Nl = static_cast<long long>(Wl) * Hl;
    const long long i = static_cast<long long>(gy) * Wl + gx;
    const float mx = __ldcs(mv + i), my = __ldcs(mv + Nl + i);
    const float ix = fminf(fmaxf(floorf(mx), -1048576.0f), 1048576.0f);
    const float iy = fminf(fmaxf(floorf(my), -1048576.0f), 1048576.0f);
    float fx = mx - floorf(mx), fy = my - floorf(my);
    int X0 = gx + static_cast<int>(ix), Y0 = gy + static_cast<int>(iy);
    if (X0 < 0) { X0 = 0; fx = 0.0f; } else if (X0 >= Wl - 1) { X0 = Wl - 1; fx = 0.0f; }
    if (Y0 < 0) { Y0 = 0; fy = 0.0f; } else if (Y0 >= Hl - 1) { Y0 = Hl - 1; fy = 0.0f; }
    const int X1 = X0 + 1 < Wl ? X0 + 1 : Wl - 1;
    const int Y1 = Y0 + 1 < Hl ? Y0 + 1 : Hl - 1;
    const float *r0 = prev + static_cast<long long>(Y0) * Wl;
    const float *r1 = prev + static_cast<long long>(Y1) * Wl;
    float p[12];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        p[4 * c + 0] = __ldg(r0 + c * Nl + X0);
        p[4 * c + 1] = __ldg(r0 + c * Nl + X1);
        p[4 * c + 2] = __ldg(r1 + c * Nl + X0);
        p[4 * c + 3] = __ldg(r1 + c * Nl + X1);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        __stcs(warped + c * Nl + i, (1.0f - fy) * ((1.0f - fx) * p[4 * c] + fx * p[4 * c + 1]) +
                                        fy * ((1.0f - fx) * p[4 * c + 2] + fx * p[4 * c + 3]));
}

// ------------------------------------------------------------ host side
// 3-D FP32 map over planar [planes][H][W] with a box (bx, by, bz).
bool make_map(CUtensorMap *map, const float *base, int W, int H, int planes, int bx, int by,
              int bz) {
    auto fn = tensor_map_encoder();
    if (!fn) return false;
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(W), static_cast<cuuint64_t>(H),
                          static_cast<cuuint64_t>(planes)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(W) * 4ull,
                             static_cast<cuuint64_t>(W) * static_cast<cuuint64_t>(H) * 4ull};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(bx), static_cast<cuuint32_t>(by),
                         static_cast<cuuint32_t>(bz)};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int C, bool UP, bool TEMP, bool TONE, int NS>
int launch_variant(const CUtensorMap &ml, const CUtensorMap &mn, const CUtensorMap &mw,
                   const CUtensorMap &mc, const uint8_t *mask, int Wl, int Hl, float *out,
                   float *out_ldr, const ToneArgs &tm, int32_t *status, int stall_tile,
                   cudaStream_t stream) {
    using S = Stage<C, UP, TEMP>;
    const size_t smem =
        128 + 256 + static_cast<size_t>(NS) * S::kFloats * 4u + 2u * 5u * kPixels * sizeof(float);
    auto kern = recon_tma_kernel<C, UP, TEMP, TONE, NS>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
        return SPP_ERR_CUDA;
    TileGeom g;
    g.tiles_x = (Wl + kPX - 1) / kPX;
    const int tiles_y = (Hl + kPY - 1) / kPY;
    g.num_tiles = g.tiles_x * tiles_y;
    int grid = sm_count();
    if (grid > g.num_tiles) grid = g.num_tiles;
    launch_dependent(kern, dim3(grid), dim3(kThreads), smem, stream, ml, mn, mw, mc, mask, Wl, Hl,
                     g, out, out_ldr, tm, status, stall_tile);
    count_launch();
    return launch_status();
}

}  // namespace

void launch_warp_prev(const float *prev, const float *mv, int Wl, int Hl, float *warped,
                      cudaStream_t stream) {
    dim3 grid((Wl + 63) / 64, (Hl + 3) / 4);
    warp_prev_kernel<<<grid, 256, 0, stream>>>(prev, mv, Wl, Hl, warped);
}

bool launch_recon_tma(const float *noisy, const float *logits, int C_total, int C_used,
                      const float *coarse, const float *warped, const uint8_t *mask, int Wl,
                      int Hl, float *out, float *out_ldr, const ToneArgs &tm, int32_t *status,
                      cudaStream_t stream, int *rc) {
    *rc = SPP_OK;
    if ((Wl % 4) != 0 || Wl < 8 || Hl < 4) return false;
    if (C_used != 25 && C_used != 29 && C_used != 54) return false;
    const bool up = coarse != nullptr, temp = warped != nullptr;
    if (temp && (!up || C_used != 54)) return false;
    if (!temp && C_used == 54) return false;
    if (!up && C_used != 25) return false;
    if (up && !temp && C_used != 29) return false;
    // the coarse level's map needs 16-byte row strides
    if (up && (((Wl >> 1) % 4) != 0 || !aligned16(coarse))) return false;
    CUtensorMap ml, mn, mw, mc;
    if (!make_map(&ml, logits, Wl, Hl, C_total, kPX, kPY, C_used)) return false;
    if (!make_map(&mn, noisy, Wl, Hl, 3, kBoxX, kBoxY, 3)) return false;
    if (temp) {
        if (!make_map(&mw, warped, Wl, Hl, 3, kBoxX, kBoxY, 3)) return false;
    } else {
        mw = mn;  // unused
    }
    if (up) {
        if (!make_map(&mc, coarse, Wl >> 1, Hl >> 1, 3, kCoarseX, kCoarseY, 3)) return false;
    } else {
        mc = mn;  // unused
    }
    const bool tone = out_ldr != nullptr;
    const int stall = g_recon_stall_tile.exchange(-1);
    if (temp) {
        *rc = tone ? launch_variant<54, true, true, true, 3>(ml, mn, mw, mc, mask, Wl, Hl, out,
                                                             out_ldr, tm, status, stall, stream)
                   : launch_variant<54, true, true, false, 3>(ml, mn, mw, mc, mask, Wl, Hl, out,
                                                              out_ldr, tm, status, stall, stream);
    } else if (up) {
        *rc = tone ? launch_variant<29, true, false, true, 5>(ml, mn, mw, mc, mask, Wl, Hl, out,
                                                              out_ldr, tm, status, stall, stream)
                   : launch_variant<29, true, false, false, 5>(ml, mn, mw, mc, mask, Wl, Hl,
                                                               out, out_ldr, tm, status, stall, stream);
    } else {
        *rc = tone ? launch_variant<25, false, false, true, 5>(ml, mn, mw, mc, mask, Wl, Hl,
                                                               out, out_ldr, tm, status, stall, stream)
                   : launch_variant<25, false, false, false, 5>(ml, mn, mw, mc, mask, Wl, Hl,
                                                                out, out_ldr, tm, status, stall, stream);
    }
    return true;
}

}  // namespace spp
