// 3x3 convolution (zero padding, stride 1) as an implicit GEMM on the
// tcgen05 tensor cores: BF16 operands, FP32 accumulation in TMEM.
//
// GEMM view: M = 128 output pixels of one image row, N = output channels,
// K = 9 taps x input channels.  One CTA per SM runs persistently over
// tiles of TR rows x 128 pixels; the accumulator of each row is an
// M=128 x N block of TMEM columns, double-buffered across tiles so the
// epilogue of one tile overlaps the main loop of the next.
//
// Warp roles (320 threads):
//   warps 0-3  epilogue: tcgen05.ld of the accumulator (warp w reads TMEM
//              lanes 32w..32w+31 = pixels), bias / ReLU / mask, stores;
//   warps 4-7  a second set of epilogue warps (the second half of each
//              tile's rows, TMEM lanes 32 (w - 4)..) when the input arrives by
//              TMA and N <= 64, with warp 9 issuing the copies; otherwise
//              producers: per K chunk of 16 input channels they stage the
//              (TR+2) x 130 pixel halo of the tile in shared memory as K-major
//              rows of 32 bytes per pixel in the 32-byte swizzle ([row][pixel]
//              [16 ch], a_off), with zero padding, fused 2x2 pooling, fused
//              upsample + concat or FP32 -> BF16 conversion on the way (a TMA
//              box writes the plain NHWC case directly); one elected thread
//              bulk-copies the pre-packed weights of the chunk;
//   warp 8     lane 0 issues the MMAs: for each row r and tap (dy, dx) the A
//              operand is the halo window starting at row r+dy, pixel dx
//              (a start address moved by whole 32-byte pixel rows, which the
//              swizzled descriptor allows because the swizzle follows the
//              absolute address), the B operand the tap's weight block.  No
//              im2col copy is made.
//
// Stages are recycled through full/empty mbarriers (producers -> MMA via
// arrival counts and transaction bytes, MMA -> producers via
// tcgen05.commit).  Every wait is bounded: on expiry the CTA records
// SPP_ERR_TIMEOUT in the status word, the other roles leave at their next
// wait, the MMA thread waits for its issued MMAs, the copy thread for its
// copies in flight, and TMEM is freed before the kernel returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "conv_src.cuh"
#include "conv_tc.cuh"
#include "spp_internal.cuh"
#include "tc_common.cuh"
#include "tma_host.cuh"

namespace spp {
namespace conv {
namespace {

constexpr int kTileX = 128;  // output pixels per row tile (MMA M)
constexpr int kPitch = 130;  // staged halo pixels per row
constexpr int kThreads = 320;
constexpr int kHeader = 384;  // barriers, TMEM slot, abort flag
constexpr int kUpW = kTileX / 2 + 2;  // coarse pixels under a tile's halo (upsampling layers)
constexpr int kSmemLimit = 227 * 1024;             // dynamic shared memory per CTA
constexpr int kSmemBudget = kSmemLimit - 512;      // minus alignment slack

constexpr int kResidentMax = 80 * 1024;  // weights kept in shared memory up to this size

// RES: all weights of the layer stay resident in shared memory (loaded once
// per CTA); otherwise each stage carries its chunk's weights.
template <int N, bool RES>
struct Cfg {
    static constexpr int TR = N <= 64 ? 4 : N <= 128 ? 2 : 1;  // rows per tile
    // halo bytes per stage: (TR+2) x 130 pixel rows of 32 bytes (16 channels),
    // 32-byte swizzled (a_off), a multiple of the 256-byte swizzle period
    static constexpr int kA = ((TR + 2) * kPitch * 32 + 255) / 256 * 256;
    static constexpr int kB = 9 * 2 * N * 16;                   // weight bytes per K chunk
    static constexpr int kStage = RES ? kA : kA + kB;
    static constexpr int kWRegion = RES ? kResidentMax : 0;
    static constexpr int kEpiBytes = RES ? 4 * 2 * (N >= 32 ? 32 : 16) * 32 * 4 : 0;
    static constexpr int kBiasOff = kHeader;                     // FP32 bias [N]
    static constexpr int kZeroOff = kBiasOff + 1024;             // zero operand (stacked)
    // N = 32 and 64: the three dy taps of a halo row are one MMA of 3 N columns
    // whose output spans three neighbouring output rows (below)
    static constexpr bool kStack = (N == 32 || N == 64);
    // rows of the zero operand that resets the TR accumulator rows (at least
    // the 128 rows of the A side), in both 8-channel groups
    static constexpr int kZeroRows = TR * N > 128 ? TR * N : 128;
    static constexpr int kZeroBytes = kStack ? 2 * kZeroRows * 16 : 0;
    static constexpr int kWOff = kZeroOff + kZeroBytes;          // resident weights
    static constexpr int kStagesOff = (kWOff + kWRegion + 255) / 256 * 256;
    // BF16 NHWC outputs leave through a per-warp staging row buffer, so that
    // each warp store writes contiguous 512-byte runs ([32 px][kCBs ch] with
    // a 16-byte pad per pixel: conflict-free 16-byte shared accesses)
    static constexpr int kCBs = N < 32 ? N : 32;
    static constexpr int kStageRow = 2 * kCBs + 16;
    // eight epilogue warps (two per TMEM sub-partition, each taking half of
    // a tile's rows) when the layer's input comes by TMA and N <= 64, else four
    static constexpr int kEpiWarps = N <= 64 ? 8 : 4;
    static constexpr int kStoreBytes = kEpiWarps * 32 * kStageRow;
    // the FP32 planar staging buffers and the BF16 staging rows share one
    // region (a launch uses one of the two epilogues)
    static constexpr int kOutBytes = kEpiBytes > kStoreBytes ? kEpiBytes : kStoreBytes;
    static constexpr int kNS0 = (kSmemBudget - kStagesOff - kOutBytes) / kStage;
    static constexpr int kNS = kNS0 > 8 ? 8 : kNS0;
    // a stage is published kLag stages after its copies were issued; kLag <=
    // kNS - 2 lets the MMAs of one stage run while the next is published
    static constexpr int kLag = kNS - 2;
    // Stacked MMAs: halo row h feeds output rows h - 2, h - 1, h (dy = 2, 1,
    // 0); the first two and the last two halo rows of a tile feed only the
    // output rows inside the tile, through the matching part of the stacked
    // weights, so each accumulator holds exactly the TR rows; one 0 x 0 MMA
    // with accumulate off resets them at the start of a tile, after which
    // every MMA accumulates
    static constexpr int kRowOff = 0;
    static constexpr int kAccCols = TR * N;
    static constexpr int kCols = tc::pow2_cols(2 * kAccCols);
    static_assert(2 * kAccCols <= 512, "accumulators exceed TMEM");
    // FP32 planar outputs leave through two 8 KB staging buffers ([16 ch][128 px])
    // and TMA tensor stores (resident-weight variants; the heads are)
    static constexpr int kEpiOff = (kStagesOff + kNS * kStage + 127) / 128 * 128;
    static constexpr int kStoreOff = kEpiOff;
    static constexpr int kSmem = kEpiOff + kOutBytes + 256;  // + alignment slack
    // Upsampling layers (tma_in == 3): the coarse rows under a tile's halo,
    // one TMA box of 16 channels, in two buffers after the other areas (when
    // they fit): [buffer 2][kUpRows][kUpW][16 ch], not swizzled
    static constexpr int kUpRows = TR / 2 + 2;
    static constexpr int kUpBox = kUpRows * kUpW * 32;         // bytes of one box
    static constexpr int kUpG = (kUpBox + 127) / 128 * 128;     // its 128-byte aligned slot
    static constexpr int kUpOff = (kStoreOff + kStoreBytes + 127) / 128 * 128;
    // (upsampling layers have BF16 outputs: the buffers may overlap the FP32 area)
    static constexpr int kSmemUp0 = kUpOff + 2 * kUpG + 256;
    static constexpr int kSmemUp = kSmemUp0 > kSmem ? kSmemUp0 : kSmem;
    static constexpr bool kUpFits = kSmemUp <= kSmemLimit;
    static_assert(kSmem <= kSmemLimit, "shared memory over the per-CTA limit");
    static_assert(kNS >= 2, "stage does not fit twice");
};

struct Bars {
    uint64_t full[8];   // producers' halo stores (128 arrivals)
    uint64_t wfull[8];  // weight bulk copies (1 arrival + bytes); [0] only when resident
    uint64_t empty[8];  // MMA done with the stage (tcgen05.commit)
    uint64_t accf[2];   // accumulator ready (tcgen05.commit)
    uint64_t acce[2];   // accumulator drained by the epilogue (128 arrivals)
    uint64_t drain;     // abort path: all issued MMAs complete
    uint64_t upfull[2]; // coarse boxes of an upsampling layer landed (1 arrival + bytes)
    uint64_t updone[2]; // coarse buffer expanded by every producer (160 arrivals)
    uint32_t tmem_base;
    int abort;
};
static_assert(sizeof(Bars) <= kHeader, "header");

// Byte offset in a stage of the 8 channels kg (0, 1) of halo pixel (row, px):
// rows of 32 bytes (one 16-channel K chunk) in the K-major 32-byte swizzle
// (the 16-byte half kg of row q sits at half kg ^ bit 2 of q), the layout a
// TMA box with CU_TENSOR_MAP_SWIZZLE_32B writes to a 256-byte aligned stage
// and the one the MMA reads through a SWIZZLE_32B descriptor at any row start
__device__ __forceinline__ int a_off(int row, int px, int kg) {
    const int q = row * kPitch + px;
    return q * 32 + 16 * (kg ^ ((q >> 2) & 1));
}


// TMA load of an NHWC halo box [1 group][TR+2 rows][130 px][8 ch] (5-D map:
// channel-in-group, x, y, group, image) into shared memory, completing on bar.
__device__ __forceinline__ void tma_load_halo(const CUtensorMap *map, void *dst, uint64_t *bar,
                                              int x, int y, int g, int b) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(tc::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(tc::smem_u32(bar)), "r"(0), "r"(x), "r"(y),
        "r"(g), "r"(b)
        : "memory");
}

// TMA tensor store of a [16][1][128] FP32 box from shared memory at (x, y, c, b).
__device__ __forceinline__ void tma_store_planes(const CUtensorMap *map, const void *src, int x,
                                                 int y, int c, int b) {
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(tc::smem_u32(src)), "r"(x), "r"(y), "r"(c), "r"(b)
        : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// the stores committed before the last `pending` have finished reading shared memory
template <int P>
__device__ __forceinline__ void tma_store_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(P) : "memory");
}
__device__ __forceinline__ void tma_store_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

template <int N, bool RES>
__global__ void __launch_bounds__(kThreads, 1) conv3x3_kernel(const ConvArgs a,
                                                             const __grid_constant__ CUtensorMap omap,
                                                             const __grid_constant__ CUtensorMap imap,
                                                             const __grid_constant__ CUtensorMap umap) {
    using C = Cfg<N, RES>;
    constexpr int TR = C::TR, NS = C::kNS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((256u - (tc::smem_u32(smem_raw) & 255u)) & 255u);
    Bars &bars = *reinterpret_cast<Bars *>(base);
    unsigned char *wres = base + C::kWOff;              // resident weights (RES)
    unsigned char *stages = base + C::kStagesOff;
    float *sbias = reinterpret_cast<float *>(base + C::kBiasOff);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int tiles_x = (a.W + kTileX - 1) / kTileX;
    const int tiles_y = (a.H + TR - 1) / TR;
    const int per_img = tiles_x * tiles_y;
    const int ntiles = a.B * per_img;
    const int kchunks = a.cin_pad / 16;

    // the second set of epilogue warps: for a plain NHWC input (TMA halo, one
    // issuing thread) the producer warps 4-7 take half of each tile's output
    // rows and warp 9 issues the copies
    const bool ep8 = C::kEpiWarps == 8 && a.tma_in == 1;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&bars.full[s], a.tma_in == 1 ? 1 : a.tma_in == 3 ? 160 : 128);
            tc::mbar_init(&bars.wfull[s], 1);
            tc::mbar_init(&bars.empty[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&bars.accf[i], 1);
            tc::mbar_init(&bars.acce[i], ep8 ? 256 : 128);
        }
        tc::mbar_init(&bars.drain, 1);
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&bars.upfull[i], 1);
            tc::mbar_init(&bars.updone[i], 160);
        }
        bars.abort = 0;
        tc::fence_mbar_init();
    }
    if (C::kStack) {
        // the zero operand that resets an accumulator (0 x 0 with accumulate off)
        for (int i = tid; i < C::kZeroBytes / 16; i += kThreads)
            reinterpret_cast<uint4 *>(base + C::kZeroOff)[i] = make_uint4(0, 0, 0, 0);
        tc::fence_proxy_async();
    }
    if (warp == 8) tc::tmem_alloc(&bars.tmem_base, C::kCols);
    // launched as a programmatic dependent: the set-up above touches no global
    // memory; every global access below comes after the previous kernel of the
    // stream has completed
    pdl_wait();
    pdl_trigger();
    for (int i = tid; i < N; i += kThreads) sbias[i] = (a.bias && i < a.cout) ? a.bias[i] : 0.f;
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = bars.tmem_base;
    volatile int *abort_flag = &bars.abort;
    auto fail = [&]() {
        *abort_flag = 1;
        set_status(a.status, SPP_ERR_TIMEOUT);
    };

    // producers: warps 4-7, joined by warp 9 for an upsampling layer (whose
    // expansion of the coarse boxes bounds it), or warp 9 alone (TMA-fed
    // layers with eight epilogue warps)
    const bool up5 = a.tma_in == 3;
    if (ep8 ? warp == 9 : (warp >= 4 && warp < 8) || (up5 && warp == 9)) {
        // ---------------------------------------------------------- producers
        const int ptid = ep8 ? tid - 288 : warp == 9 ? tid - 160 : tid - 128;
        const int nprod = up5 ? 160 : 128;  // threads sharing the expansion tasks
        constexpr int kTasks = 2 * (TR + 2) * kPitch;  // 16-byte chunks per stage
        constexpr int kPer = (kTasks + 127) / 128;
        // this thread's tasks (the same in every stage): row << 10 | px << 1 | kg
        int tinfo[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int j = u * nprod + ptid;
            tinfo[u] = j < kTasks ? (((j >> 1) / kPitch) << 10) | (((j >> 1) % kPitch) << 1) | (j & 1)
                                  : -1;
        }
        // upsampling layers: this thread's coarse pieces (the same in every
        // chunk): coarse row << 10 | coarse column << 1 | 8-channel half
        constexpr int kUpTasks = C::kUpRows * kUpW * 2;
        constexpr int kUpPer = (kUpTasks + 127) / 128;
        int uinfo[kUpPer];
#pragma unroll
        for (int k = 0; k < kUpPer; ++k) {
            const int j = k * nprod + ptid;
            uinfo[k] = j < kUpTasks ? (((j >> 1) / kUpW) << 10) | (((j >> 1) % kUpW) << 1) | (j & 1)
                                    : -1;
        }
        uint32_t it = 0;
        uint32_t issued = 0;  // weight copies issued (by ptid 0)
        bool ok = true;
        // Sources that need no arithmetic go through cp.async (zero-fill for
        // the padding); a stage is published NS-1 stages later, so that up to
        // NS-1 stages of copies are in flight per thread.  The other modes
        // (FP32 planar gradients of the heads, pooling on load) stage through
        // registers and publish at once.
        const bool async_src = a.src_mode == kSrcNHWC || a.src_mode == kSrcConcatUp;
        constexpr uint32_t kLag = C::kLag;
        uint32_t published = 0;
        // arrival for a cp.async stage whose copies have landed (TMA stages of
        // an upsampling layer arrived when they were issued)
        auto publish_lagged = [&](uint32_t k) {
            const int ck = static_cast<int>(k % static_cast<uint32_t>(kchunks));
            if (a.tma_in == 2 && ck * 16 < a.c0) return;
            tc::fence_proxy_async();
            tc::mbar_arrive(&bars.full[k % NS]);
        };
        // tma_in == 3: the u-th upsampled chunk of this CTA (tile blockIdx.x +
        // (u / nup) * gridDim.x, chunk c0 / 16 + u % nup) has its coarse box in
        // buffer u & 1; the box of chunk u + 1 is requested while chunk u is
        // expanded
        const int nup = a.tma_in == 3 ? kchunks - a.c0 / 16 : 0;
        uint32_t u_next = 0, u_issued = 0;
        auto issue_up = [&](uint32_t u) {  // thread ptid 0
            const int t = blockIdx.x + static_cast<int>(u / nup) * gridDim.x;
            if (t >= ntiles) return;
            const int b = t / per_img, r = t - b * per_img;
            const int y0 = (r / tiles_x) * TR, x0 = (r % tiles_x) * kTileX;
            uint64_t *bar = &bars.upfull[u & 1];
            tc::mbar_arrive_expect_tx(bar, C::kUpBox);
            tma_load_halo(&umap, base + C::kUpOff + (u & 1) * C::kUpG, bar, (x0 >> 1) - 1,
                          (y0 - 1) >> 1, static_cast<int>(u % nup), b);
            u_issued = u + 1;
        };
        if (nup > 0 && ptid == 0) issue_up(0);
        if (RES && ptid == 0) {
            // the whole packed weight operand, once
            tc::mbar_arrive_expect_tx(&bars.wfull[0], static_cast<uint32_t>(kchunks * C::kB));
            for (int c = 0; c < kchunks; ++c)
                tc::bulk_g2s(wres + c * C::kB,
                             reinterpret_cast<const unsigned char *>(a.wpack) +
                                 static_cast<size_t>(c) * C::kB,
                             C::kB, &bars.wfull[0]);
            issued = 1;
        }
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int b = t / per_img, r = t - b * per_img;
            const int y0 = (r / tiles_x) * TR, x0 = (r % tiles_x) * kTileX;
            for (int c = 0; c < kchunks; ++c) {
                const int s = static_cast<int>(it % NS);
                const uint32_t ph = (it / NS) & 1u;
                if (!tc::mbar_wait(&bars.empty[s], ph ^ 1u, abort_flag)) {
                    fail();
                    ok = false;
                    break;
                }
                unsigned char *As = stages + s * C::kStage;
                if (!RES && ptid == 0) {
                    tc::mbar_arrive_expect_tx(&bars.wfull[s], C::kB);
                    tc::bulk_g2s(As + C::kA,
                                 reinterpret_cast<const unsigned char *>(a.wpack) +
                                     static_cast<size_t>(c) * C::kB,
                                 C::kB, &bars.wfull[s]);
                    ++issued;
                }
                // task j -> 8-channel group j & 1 (fastest), then pixel, then row;
                // shared-memory offset a_off(row, px, kg)
                if (a.tma_in == 1) {
                    // the halo of both 8-channel groups as two TMA boxes (zero fill
                    // outside the image and beyond the channels)
                    if (ptid == 0) {
                        tc::mbar_arrive_expect_tx(&bars.full[s], kPitch * (TR + 2) * 32);
                        tma_load_halo(&imap, As, &bars.full[s], x0 - 1, y0 - 1, c, b);
                    }
                    ++it;
                    ++published;
                } else if (a.tma_in == 3) {
                    if (c * 16 < a.c0) {
                        // skip-connection chunk: TMA as above, every producer arrives
                        if (ptid == 0) {
                            tc::mbar_arrive_expect_tx(&bars.full[s], kPitch * (TR + 2) * 32);
                            tma_load_halo(&imap, As, &bars.full[s], x0 - 1, y0 - 1, c, b);
                        } else {
                            tc::mbar_arrive(&bars.full[s]);
                        }
                    } else {
                        // upsampled chunk: request the next chunk's coarse box once
                        // its buffer (used by chunk u_next - 1) is expanded, then
                        // expand this one: halo pixel (x, y) <- coarse (x/2, y/2),
                        // zero outside the output grid
                        const uint32_t u = u_next++;
                        if (ptid == 0) {
                            if (u >= 1 && !tc::mbar_wait(&bars.updone[(u - 1) & 1], ((u - 1) >> 1) & 1u,
                                                         abort_flag)) {
                                fail();
                                ok = false;
                                break;
                            }
                            issue_up(u + 1);
                        }
                        if (!tc::mbar_wait(&bars.upfull[u & 1], (u >> 1) & 1u, abort_flag)) {
                            fail();
                            ok = false;
                            break;
                        }
                        const unsigned char *ub = base + C::kUpOff + (u & 1) * C::kUpG;
                        // each coarse piece (cr, cx) goes to the halo rows and
                        // pixels that read it: rows 2 cr - p, 2 cr + 1 - p (p = 1
                        // when y0 is even) and pixels 2 cx - 1, 2 cx (x0 is even),
                        // those inside the halo.  W and H are even, so a halo
                        // pixel outside the image reads a coarse cell outside the
                        // coarse image, which the TMA box filled with zeros.
                        const int par = (y0 - 1) & 1;
#pragma unroll
                        for (int k = 0; k < kUpPer; ++k) {
                            if (uinfo[k] < 0) continue;
                            const int cr = uinfo[k] >> 10, cx = (uinfo[k] >> 1) & 511,
                                      kg = uinfo[k] & 1;
                            const uint4 v = *reinterpret_cast<const uint4 *>(
                                ub + (cr * kUpW + cx) * 32 + kg * 16);
#pragma unroll
                            for (int dr = 0; dr < 2; ++dr) {
                                const int row = 2 * cr + dr - par;
                                if (row < 0 || row > TR + 1) continue;
#pragma unroll
                                for (int dc = 0; dc < 2; ++dc) {
                                    const int px = 2 * cx + dc - 1;
                                    if (px < 0 || px >= kPitch) continue;
                                    *reinterpret_cast<uint4 *>(As + a_off(row, px, kg)) = v;
                                }
                            }
                        }
                        tc::fence_proxy_async();
                        tc::mbar_arrive(&bars.full[s]);
                        tc::mbar_arrive(&bars.updone[u & 1]);
                    }
                    ++it;
                    ++published;
                } else if (a.tma_in == 2 && c * 16 < a.c0) {
                    // upsampling layer, skip-connection chunk: TMA as above, every
                    // producer arrives now; an empty copy group keeps the count of
                    // groups equal to the count of stages for the lagged ones
                    if (ptid == 0) {
                        tc::mbar_arrive_expect_tx(&bars.full[s], kPitch * (TR + 2) * 32);
                        tma_load_halo(&imap, As, &bars.full[s], x0 - 1, y0 - 1, c, b);
                    } else {
                        tc::mbar_arrive(&bars.full[s]);
                    }
                    cp_async_commit();
                    ++it;
                    if (it > kLag) {
                        cp_async_wait<kLag>();
                        publish_lagged(published);
                        ++published;
                    }
                } else if (async_src) {
                    const uint32_t sbase = tc::smem_u32(As);
#pragma unroll
                    for (int u = 0; u < kPer; ++u) {
                        if (tinfo[u] < 0) continue;
                        const int row = tinfo[u] >> 10, px = (tinfo[u] >> 1) & 511, kg = tinfo[u] & 1;
                        const __nv_bfloat16 *src = chunk_address(a, b, y0 - 1 + row, x0 - 1 + px,
                                                                 c * 16 + kg * 8);
                        cp_async16(sbase + a_off(row, px, kg),
                                   src ? src : a.src0, src ? 16u : 0u);
                    }
                    cp_async_commit();
                    ++it;
                    if (it > kLag) {
                        cp_async_wait<kLag>();
                        publish_lagged(published);
                        ++published;
                    }
                } else {
                    constexpr int kUnroll = 4;
#pragma unroll 1
                    for (int j0 = 0; j0 < kTasks; j0 += 128 * kUnroll) {
                        uint4 v[kUnroll];
#pragma unroll
                        for (int u = 0; u < kUnroll; ++u) {
                            const int j = j0 + u * 128 + ptid;
                            v[u] = make_uint4(0, 0, 0, 0);
                            if (j < kTasks) {
                                const int kg = j & 1, px = (j >> 1) % kPitch, row = (j >> 1) / kPitch;
                                v[u] = load_chunk(a, b, y0 - 1 + row, x0 - 1 + px,
                                                  c * 16 + kg * 8);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kUnroll; ++u) {
                            const int j = j0 + u * 128 + ptid;
                            if (j < kTasks) {
                                const int kg = j & 1, px = (j >> 1) % kPitch, row = (j >> 1) / kPitch;
                                *reinterpret_cast<uint4 *>(As + a_off(row, px, kg)) = v[u];
                            }
                        }
                    }
                    tc::fence_proxy_async();
                    tc::mbar_arrive(&bars.full[s]);
                    ++it;
                    ++published;
                }
            }
        }
        // publish the stages still in flight (also on the abort path, where the
        // copies must land before the CTA exits)
        cp_async_wait<0>();
        for (; published < it; ++published) publish_lagged(published);
        if (!ok && ptid == 0) {
            // wait (bounded, ignoring the abort flag) for the copies still in flight
            if (a.tma_in == 1) {
                const uint32_t first = it > NS ? it - NS : 0;
                for (uint32_t k = first; k < it; ++k)
                    (void)tc::mbar_wait(&bars.full[k % NS], (k / NS) & 1u, nullptr);
            }
            if (a.tma_in >= 2) {
                // the skip-connection boxes (TMA) among the last stages
                const uint32_t first = it > NS ? it - NS : 0;
                for (uint32_t k = first; k < it; ++k)
                    if (static_cast<int>(k % static_cast<uint32_t>(kchunks)) * 16 < a.c0)
                        (void)tc::mbar_wait(&bars.full[k % NS], (k / NS) & 1u, nullptr);
            }
            // coarse boxes requested (the last two, one per buffer)
            for (uint32_t k = u_issued > 2 ? u_issued - 2 : 0; k < u_issued; ++k)
                (void)tc::mbar_wait(&bars.upfull[k & 1], (k >> 1) & 1u, nullptr);
            if (RES) {
                if (issued) (void)tc::mbar_wait(&bars.wfull[0], 0, nullptr);
            } else {
                const uint32_t first = issued > NS ? issued - NS : 0;
                for (uint32_t k = first; k < issued; ++k)
                    (void)tc::mbar_wait(&bars.wfull[k % NS], (k / NS) & 1u, nullptr);
            }
        }
    } else if (warp == 8) {
        // -------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(128, N);
            constexpr uint32_t kLboB = N * 16;
            uint32_t it = 0, tl = 0;
            bool ok = true, pending = false;
            if (RES && ntiles > static_cast<int>(blockIdx.x) &&
                !tc::mbar_wait(&bars.wfull[0], 0, abort_flag)) {
                fail();
                ok = false;
            }
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
                const int acc = tl & 1;
                if (!tc::mbar_wait(&bars.acce[acc], ((tl >> 1) & 1u) ^ 1u, abort_flag)) {
                    fail();
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t d0 = tmem + acc * C::kAccCols;
                if (C::kStack) {
                    // reset the TR accumulator rows
                    const uint64_t zd = tc::smem_desc(tc::smem_u32(base + C::kZeroOff),
                                                      C::kZeroRows * 16, 128);
                    tc::mma_bf16(d0, zd, zd, tc::idesc_bf16_f32(128, TR * N), 0u);
                }
                for (int c = 0; c < kchunks; ++c, ++it) {
                    const int s = static_cast<int>(it % NS);
                    const uint32_t ph = (it / NS) & 1u;
                    if (!tc::mbar_wait(&bars.full[s], ph, abort_flag) ||
                        (!RES && !tc::mbar_wait(&bars.wfull[s], ph, abort_flag))) {
                        fail();
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t a_base = tc::smem_u32(stages + s * C::kStage);
                    const uint32_t b_base =
                        RES ? tc::smem_u32(wres + c * C::kB) : a_base + C::kA;
                    if (C::kStack) {
                        // halo row h feeds output rows h-2, h-1, h through the
                        // stacked weights [dy = 2; dy = 1; dy = 0] of its dx tap;
                        // rows outside the tile are left out (the matching part of
                        // the stacked weights, fewer MMA columns)
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
                            const uint32_t bdx = b_base + dx * 2 * 3 * N * 16;
#pragma unroll
                            for (int h = 0; h < TR + 2; ++h) {
                                const int rlo = h - 2 < 0 ? 0 : h - 2;   // first row fed
                                const int rhi = h < TR - 1 ? h : TR - 1;  // last row fed
                                const int k0 = rlo - (h - 2);             // its dy block
                                const uint64_t bd =
                                    tc::smem_desc(bdx + k0 * N * 16, 3 * N * 16, 128);
                                const uint64_t ad =
                                    tc::smem_desc_sw32(a_base + (h * kPitch + dx) * 32);
                                tc::mma_bf16(d0 + rlo * N, ad, bd,
                                             tc::idesc_bf16_f32(128, (rhi - rlo + 1) * N), 1u);
                            }
                        }
                    } else {
#pragma unroll
                        for (int tap = 0; tap < 9; ++tap) {
                            const int dy = tap / 3, dx = tap % 3;
                            const uint64_t bd =
                                tc::smem_desc(b_base + tap * 2 * N * 16, kLboB, 128);
#pragma unroll
                            for (int r = 0; r < TR; ++r) {
                                const uint64_t ad =
                                    tc::smem_desc_sw32(a_base + ((r + dy) * kPitch + dx) * 32);
                                tc::mma_bf16(d0 + r * N, ad, bd, idesc, (c | tap) != 0);
                            }
                        }
                    }
                    pending = true;
                    tc::mma_commit(&bars.empty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&bars.accf[acc]);
            }
            if (!ok && pending) {
                tc::mma_commit(&bars.drain);
                (void)tc::mbar_wait(&bars.drain, 0, nullptr);
            }
        }
        __syncwarp();
    } else if (warp < 4 || (ep8 && warp < 8)) {
        // ----------------------------------------------------------- epilogue
        // warp w reads TMEM lanes 32 (w % 4) ..; with eight epilogue warps,
        // warps 0-3 take the first half of a tile's rows and 4-7 the second
        const int sub = warp & 3;
        const int row_lo = ep8 ? (warp >> 2) * (TR / 2) : 0;
        const int row_hi = ep8 ? row_lo + TR / 2 : TR;
        uint32_t tl = 0;
        uint32_t eblk = 0;  // TMA-stored blocks (planar outputs)
        const uint32_t lane_base = static_cast<uint32_t>(sub * 32) << 16;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
            const int acc = tl & 1;
            if (!tc::mbar_wait(&bars.accf[acc], (tl >> 1) & 1u, abort_flag)) {
                fail();
                break;
            }
            tc::tc_fence_after();
            const int b = t / per_img, rr = t - b * per_img;
            const int y0 = (rr / tiles_x) * TR, x = (rr % tiles_x) * kTileX + sub * 32 + lane;
            const uint32_t abase = tmem + lane_base + acc * C::kAccCols + C::kRowOff * N;
            // hands the accumulator back to the MMA warp
            auto release_acc = [&]() {
                tc::tc_fence_before();
                tc::mbar_arrive(&bars.acce[acc]);
            };
            if (TR % 2 == 0 && a.pool_out) {
                // ReLU rows in pairs, plus the 2x2 average of their BF16 values
                // (lanes x and x^1 hold horizontal neighbours), up to 32 columns
                // of both rows per TMEM round trip; each of the two rows and the
                // pooled row leaves through the warp's staging row buffer as
                // contiguous runs
                constexpr int kCB = N < 32 ? N : 32;
                constexpr int kW = kCB / 2;  // packed BF16 pairs per pixel and block
                unsigned char *srow = base + C::kStoreOff + (warp * 32) * C::kStageRow;
                const int xw = x - lane;     // the warp's first pixel
                // stages kW words per lane (or per listed pixel) and writes the
                // pixels [0, npx) of the staging rows as 16-byte chunks to dst
                auto flush = [&](int npx, auto valid, auto address) {
                    __syncwarp();
                    constexpr int kChunks = kCB / 8;
#pragma unroll
                    for (int i = 0; i < kChunks; ++i) {
                        const int pp = i * (32 / kChunks) + lane / kChunks;
                        const int ch = lane % kChunks;
                        if (pp < npx && valid(pp)) {
                            const uint4 val = *reinterpret_cast<const uint4 *>(
                                srow + pp * C::kStageRow + 16 * ch);
                            *reinterpret_cast<uint4 *>(address(pp) + 8 * ch) = val;
                        }
                    }
                    __syncwarp();
                };
#pragma unroll 1
                for (int r = row_lo; r < row_hi; r += 2) {
                    const int y = y0 + r;
#pragma unroll 1
                    for (int j0 = 0; j0 < N; j0 += kCB) {
                        uint32_t v0[kCB], v1[kCB];
#pragma unroll
                        for (int q = 0; q < kCB / 16; ++q) {
                            tc::tmem_ld16(abase + r * N + j0 + 16 * q,
                                          *reinterpret_cast<uint32_t(*)[16]>(v0 + 16 * q));
                            tc::tmem_ld16(abase + (r + 1) * N + j0 + 16 * q,
                                          *reinterpret_cast<uint32_t(*)[16]>(v1 + 16 * q));
                        }
                        tc::tmem_wait_ld();
                        uint32_t w1[kW], wp[kW];
#pragma unroll
                        for (int e = 0; e < kCB; e += 2) {
                            float f0[2], f1[2], sm[2];
#pragma unroll
                            for (int t = 0; t < 2; ++t) {
                                const float bb = sbias[j0 + e + t];
                                f0[t] = __bfloat162float(__float2bfloat16_rn(
                                    fmaxf(__uint_as_float(v0[e + t]) + bb, 0.f)));
                                f1[t] = __bfloat162float(__float2bfloat16_rn(
                                    fmaxf(__uint_as_float(v1[e + t]) + bb, 0.f)));
                                sm[t] = f0[t] + f1[t];
                                sm[t] += __shfl_xor_sync(0xffffffffu, sm[t], 1);
                            }
                            v0[e / 2] = pack_bf16x2(f0[0], f0[1]);  // row r, packed in place
                            w1[e / 2] = pack_bf16x2(f1[0], f1[1]);
                            wp[e / 2] = pack_bf16x2(0.25f * sm[0], 0.25f * sm[1]);
                        }
                        // row r
#pragma unroll
                        for (int q = 0; q < kW / 4; ++q)
                            reinterpret_cast<uint4 *>(srow + lane * C::kStageRow)[q] =
                                make_uint4(v0[4 * q], v0[4 * q + 1], v0[4 * q + 2], v0[4 * q + 3]);
                        flush(32, [&](int pp) { return xw + pp < a.W && y < a.H; },
                              [&](int pp) {
                                  return a.out +
                                         ((static_cast<size_t>(b) * a.H + y) * a.W + xw + pp) * N + j0;
                              });
                        // row r + 1
#pragma unroll
                        for (int q = 0; q < kW / 4; ++q)
                            reinterpret_cast<uint4 *>(srow + lane * C::kStageRow)[q] =
                                make_uint4(w1[4 * q], w1[4 * q + 1], w1[4 * q + 2], w1[4 * q + 3]);
                        flush(32, [&](int pp) { return xw + pp < a.W && y + 1 < a.H; },
                              [&](int pp) {
                                  return a.out + ((static_cast<size_t>(b) * a.H + y + 1) * a.W +
                                                  xw + pp) * N + j0;
                              });
                        // the pooled row: pixel pair k (lanes 2k, 2k+1) at staging row k
                        if (!(lane & 1)) {
#pragma unroll
                            for (int q = 0; q < kW / 4; ++q)
                                reinterpret_cast<uint4 *>(srow + (lane >> 1) * C::kStageRow)[q] =
                                    make_uint4(wp[4 * q], wp[4 * q + 1], wp[4 * q + 2], wp[4 * q + 3]);
                        }
                        flush(16, [&](int pp) { return xw + 2 * pp + 1 < a.W + 1 &&
                                                       xw + 2 * pp < a.W && y + 1 < a.H; },
                              [&](int pp) {
                                  return a.pool_out +
                                         ((static_cast<size_t>(b) * (a.H >> 1) + (y >> 1)) *
                                              (a.W >> 1) + (xw >> 1) + pp) * N + j0;
                              });
                    }
                }
                release_acc();
                continue;
            }
            if (RES && a.epi_mode == kEpiF32Planar && a.tma_out) {
                // each epilogue warp stages kPB output planes of its 32 pixels of
                // the row in its own buffer and stores them with one TMA tensor
                // store (clipped at W and at cout); two buffers per warp, one
                // when eight warps share the staging area
                constexpr int kPB = N >= 32 ? 32 : 16;  // planes per block
                float *ebuf = reinterpret_cast<float *>(base + C::kEpiOff);
                const int x0 = (rr % tiles_x) * kTileX;
                constexpr int kRowBlocks = N / kPB;
                constexpr int kBlocks = TR * kRowBlocks;
                auto tmem_read = [&](int k, uint32_t (&vv)[kPB]) {
#pragma unroll
                    for (int q = 0; q < kPB / 16; ++q)
                        tc::tmem_ld16(abase + (k / kRowBlocks) * N + (k % kRowBlocks) * kPB + 16 * q,
                                      *reinterpret_cast<uint32_t(*)[16]>(vv + 16 * q));
                };
                auto pblocks = [&](auto count_c, int kb_lo) {
                    constexpr int kCount = decltype(count_c)::value;
                    uint32_t fbuf[2][kPB];
                    tmem_read(kb_lo, fbuf[0]);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int kk = 0; kk < kCount; ++kk) {
                        const int kb = kb_lo + kk;
                        if (kk + 1 < kCount) tmem_read(kb + 1, fbuf[(kk + 1) & 1]);
                        const uint32_t (&v)[kPB] = fbuf[kk & 1];
                        const int y = y0 + kb / kRowBlocks, j0 = (kb % kRowBlocks) * kPB;
                        if (j0 < a.cout) {  // padding columns are not stored
                            float *buf = ebuf + (ep8 ? warp : warp * 2 + static_cast<int>(eblk & 1)) *
                                                    kPB * 32;
                            if (lane == 0) {
                                if (ep8)
                                    tma_store_wait_read<0>();
                                else
                                    tma_store_wait_read<1>();
                            }
                            __syncwarp();
#pragma unroll
                            for (int e = 0; e < kPB; ++e)
                                buf[e * 32 + lane] = __uint_as_float(v[e]) + sbias[j0 + e];
                            tc::fence_proxy_async();
                            __syncwarp();
                            if (lane == 0 && y < a.H && x0 + sub * 32 < a.W)
                                tma_store_planes(&omap, buf, x0 + sub * 32, y, j0, b);
                            ++eblk;
                        }
                        tc::tmem_wait_ld();
                    }
                };
                if (ep8)
                    pblocks(std::integral_constant<int, kBlocks / 2>{}, row_lo * kRowBlocks);
                else
                    pblocks(std::integral_constant<int, kBlocks>{}, 0);
                release_acc();
                continue;
            }
            // one row at a time, up to 32 columns per TMEM round trip; the
            // next block's TMEM read is in flight while this one is stored
            // (tcgen05.wait::ld waits for every outstanding read, so each
            // wait covers exactly the one issued before the stores)
            constexpr int kCB = N < 32 ? N : 32;
            constexpr int kRowBlocks = N / kCB;
            constexpr int kBlocks = TR * kRowBlocks;
            auto tmem_read = [&](int k, uint32_t (&vv)[kCB]) {
                const int r = k / kRowBlocks, j0 = (k % kRowBlocks) * kCB;
#pragma unroll
                for (int q = 0; q < kCB / 16; ++q)
                    tc::tmem_ld16(abase + r * N + j0 + 16 * q,
                                  *reinterpret_cast<uint32_t(*)[16]>(vv + 16 * q));
            };
            // blocks [kb_lo, kb_lo + kCount) of the tile (kCount a constant, so
            // that the double buffer stays in registers)
            auto blocks = [&](auto count_c, int kb_lo) {
                constexpr int kCount = decltype(count_c)::value;
                uint32_t vbuf[2][kCB];
                tmem_read(kb_lo, vbuf[0]);
                tc::tmem_wait_ld();
#pragma unroll
                for (int kk = 0; kk < kCount; ++kk) {
                    const int kb = kb_lo + kk;
                    if (kk + 1 < kCount) tmem_read(kb + 1, vbuf[(kk + 1) & 1]);
                    const uint32_t (&v)[kCB] = vbuf[kk & 1];
                    const int r = kb / kRowBlocks, j0 = (kb % kRowBlocks) * kCB;
                    const int y = y0 + r;
                    const bool inside = (x < a.W) && (y < a.H);
                    const size_t pix = (static_cast<size_t>(b) * a.H + y) * a.W + x;
                    if (a.epi_mode == kEpiF32Planar) {
                        if (inside) {
                            const size_t plane = static_cast<size_t>(a.H) * a.W;
                            float *o = a.outf + static_cast<size_t>(b) * a.cout * plane +
                                       static_cast<size_t>(y) * a.W + x;
#pragma unroll
                            for (int e = 0; e < kCB; ++e) {
                                const int n = j0 + e;
                                if (n < a.cout) __stcs(o + n * plane, __uint_as_float(v[e]) + sbias[n]);
                            }
                        }
                    } else {
                        // BF16 values of this pixel's kCB channels into the warp's
                        // staging row
                        unsigned char *srow = base + C::kStoreOff + (warp * 32) * C::kStageRow;
#pragma unroll
                        for (int q = 0; q < kCB / 16; ++q) {
                            const int j = j0 + 16 * q;
                            float f[16];
#pragma unroll
                            for (int e = 0; e < 16; ++e) f[e] = __uint_as_float(v[16 * q + e]);
                            if (a.epi_mode == kEpiReluBF16 || a.epi_mode == kEpiBF16) {
#pragma unroll
                                for (int e = 0; e < 16; ++e) f[e] += sbias[j + e];
                                if (a.epi_mode == kEpiReluBF16) {
#pragma unroll
                                    for (int e = 0; e < 16; ++e) f[e] = fmaxf(f[e], 0.f);
                                }
                            } else if (a.epi_mode == kEpiMaskBF16) {
                                const uint4 *m = reinterpret_cast<const uint4 *>(a.act + pix * N + j);
#pragma unroll
                                for (int h = 0; h < 2; ++h) {
                                    const uint4 qq = inside ? __ldg(m + h) : make_uint4(0, 0, 0, 0);
                                    const uint32_t *u = &qq.x;
#pragma unroll
                                    for (int k = 0; k < 4; ++k) {
                                        const float2 mv = unpack_bf16x2(u[k]);
                                        f[8 * h + 2 * k] = mv.x > 0.f ? f[8 * h + 2 * k] : 0.f;
                                        f[8 * h + 2 * k + 1] = mv.y > 0.f ? f[8 * h + 2 * k + 1] : 0.f;
                                    }
                                }
                            }
                            uint4 *d4 = reinterpret_cast<uint4 *>(srow + lane * C::kStageRow + 32 * q);
                            d4[0] = make_uint4(pack_bf16x2(f[0], f[1]), pack_bf16x2(f[2], f[3]),
                                               pack_bf16x2(f[4], f[5]), pack_bf16x2(f[6], f[7]));
                            d4[1] = make_uint4(pack_bf16x2(f[8], f[9]), pack_bf16x2(f[10], f[11]),
                                               pack_bf16x2(f[12], f[13]), pack_bf16x2(f[14], f[15]));
                        }
                        __syncwarp();
                        // the warp's 32 pixels x kCB channels as contiguous 16-byte
                        // chunks: kCB / 8 chunks per pixel, one warp store per 32 chunks
                        constexpr int kChunks = kCB / 8;
                        const int xw = x - lane;  // the warp's first pixel
#pragma unroll
                        for (int i = 0; i < kChunks; ++i) {
                            const int pp = i * (32 / kChunks) + lane / kChunks;
                            const int ch = lane % kChunks;
                            const uint4 val =
                                *reinterpret_cast<const uint4 *>(srow + pp * C::kStageRow + 16 * ch);
                            if (xw + pp < a.W && y < a.H) {
                                const size_t q = (static_cast<size_t>(b) * a.H + y) * a.W + xw + pp;
                                *reinterpret_cast<uint4 *>(a.out + q * N + j0 + 8 * ch) = val;
                            }
                        }
                        __syncwarp();  // the staging row is rewritten by the next block
                    }
                    tc::tmem_wait_ld();
                }
            };
            if (ep8)
                blocks(std::integral_constant<int, kBlocks / 2>{}, row_lo * kRowBlocks);
            else
                blocks(std::integral_constant<int, kBlocks>{}, 0);
            release_acc();
        }
        if (lane == 0 && eblk) tma_store_wait_all();
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, C::kCols);
    }
}

__global__ void pack_weights_kernel(const float *__restrict__ w, int cin, int cout, int transpose,
                                    int cin_pad, int n, __nv_bfloat16 *__restrict__ dst) {
    const int64_t total = static_cast<int64_t>(cin_pad / 16) * 9 * 2 * n * 8;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int e = static_cast<int>(idx % 8);
        int o, kg, c, dy, dx;
        if (n == 32 || n == 64) {
            // stacked: [chunk][dx][kg][3 n = (dy = 2, 1, 0) x n][8]
            const int64_t S = 3 * static_cast<int64_t>(n);
            const int n3 = static_cast<int>((idx / 8) % S);
            kg = static_cast<int>((idx / (8 * S)) % 2);
            dx = static_cast<int>((idx / (16 * S)) % 3);
            c = static_cast<int>(idx / (48 * S));
            o = n3 % n;
            dy = 2 - n3 / n;
        } else {
            // [chunk][tap][kg][n][8]
            o = static_cast<int>((idx / 8) % n);
            kg = static_cast<int>((idx / (8 * n)) % 2);
            const int tap = static_cast<int>((idx / (16 * n)) % 9);
            c = static_cast<int>(idx / (144 * static_cast<int64_t>(n)));
            dy = tap / 3;
            dx = tap % 3;
        }
        const int k = c * 16 + kg * 8 + e;  // input channel of this convolution
        float v = 0.f;
        if (!transpose) {
            if (o < cout && k < cin) v = w[((static_cast<int64_t>(o) * cin + k) * 3 + dy) * 3 + dx];
        } else {  // data gradient: input channel k is an output channel of w
            if (o < cin && k < cout)
                v = w[((static_cast<int64_t>(k) * cin + o) * 3 + (2 - dy)) * 3 + (2 - dx)];
        }
        dst[idx] = __float2bfloat16_rn(v);
    }
}

// SPP_CONV_NO_TMA_IN=1 selects the cp.async halo producers instead of TMA
// (comparison and fallback).
bool getenv_disable_tma_in() {
    static const bool off = [] {
        const char *v = getenv("SPP_CONV_NO_TMA_IN");
        return v && v[0] == '1';
    }();
    return off;
}

template <int N, bool RES>
int launch_variant(const ConvArgs &a, cudaStream_t stream) {
    using C = Cfg<N, RES>;
    static int configured_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        if (cudaFuncSetAttribute(conv3x3_kernel<N, RES>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 C::kUpFits ? C::kSmemUp : C::kSmem) != cudaSuccess)
            return SPP_ERR_CUDA;
        configured_dev = dev;
    }
    const int64_t ntiles = static_cast<int64_t>(a.B) * ((a.H + C::TR - 1) / C::TR) *
                           ((a.W + kTileX - 1) / kTileX);
    if (ntiles == 0) return SPP_OK;
    const int grid = static_cast<int>(std::min<int64_t>(ntiles, sm_count()));
    CUtensorMap omap;
    memset(&omap, 0, sizeof(omap));
    ConvArgs b = a;
    b.tma_out = 0;
    if (RES && a.epi_mode == kEpiF32Planar && a.W % 4 == 0) {
        // [B][cout][H][W] FP32 as a 4-D tensor (x, y, plane, image), box 128 x 1 x 16 x 1
        auto enc = tensor_map_encoder();
        cuuint64_t dims[4] = {static_cast<cuuint64_t>(a.W), static_cast<cuuint64_t>(a.H),
                              static_cast<cuuint64_t>(a.cout), static_cast<cuuint64_t>(a.B)};
        cuuint64_t strides[3] = {static_cast<cuuint64_t>(a.W) * 4ull,
                                 static_cast<cuuint64_t>(a.W) * a.H * 4ull,
                                 static_cast<cuuint64_t>(a.W) * a.H * a.cout * 4ull};
        cuuint32_t box[4] = {32, 1, static_cast<cuuint32_t>(N >= 32 ? 32 : 16), 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        if (enc && enc(&omap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, a.outf, dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_NONE,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
            b.tma_out = 1;
    }
    CUtensorMap imap;
    memset(&imap, 0, sizeof(imap));
    b.tma_in = 0;
    if ((a.src_mode == kSrcNHWC || a.src_mode == kSrcConcatUp) && a.c0 % 16 == 0 &&
        !getenv_disable_tma_in()) {
        // NHWC BF16 [B][H][W][c0] as 5-D (channel in chunk, x, y, 16-channel chunk,
        // image); box 16 x 130 x (TR+2) x 1 x 1 = one K chunk of the halo, written
        // with the 32-byte swizzle of the A operand (32-byte pieces: about twice
        // the TMA throughput of 16-byte ones)
        auto enc = tensor_map_encoder();
        cuuint64_t dims[5] = {16, static_cast<cuuint64_t>(a.W), static_cast<cuuint64_t>(a.H),
                              static_cast<cuuint64_t>(a.c0 / 16), static_cast<cuuint64_t>(a.B)};
        cuuint64_t strides[4] = {static_cast<cuuint64_t>(a.c0) * 2,
                                 static_cast<cuuint64_t>(a.W) * a.c0 * 2, 32,
                                 static_cast<cuuint64_t>(a.H) * a.W * a.c0 * 2};
        cuuint32_t box[5] = {16, static_cast<cuuint32_t>(kPitch), static_cast<cuuint32_t>(C::TR + 2),
                             1, 1};
        cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        if (enc && enc(&imap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(a.src0),
                       dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
            b.tma_in = a.src_mode == kSrcNHWC ? 1 : 2;
    }
    CUtensorMap umap;
    memset(&umap, 0, sizeof(umap));
    if (b.tma_in == 2 && C::kUpFits && a.epi_mode != kEpiF32Planar && a.c1 % 16 == 0 && a.c1 > 0 && a.W % 2 == 0 &&
        a.H % 2 == 0) {
        // the coarse source [B][H/2][W/2][c1] as 5-D (channel in chunk, x, y,
        // 16-channel chunk, image); box 16 x kUpW x kUpRows x 1 x 1 = one K chunk of
        // the coarse rows under a tile's halo
        auto enc = tensor_map_encoder();
        const int Wc = a.W / 2, Hc = a.H / 2;
        cuuint64_t dims[5] = {16, static_cast<cuuint64_t>(Wc), static_cast<cuuint64_t>(Hc),
                              static_cast<cuuint64_t>(a.c1 / 16), static_cast<cuuint64_t>(a.B)};
        cuuint64_t strides[4] = {static_cast<cuuint64_t>(a.c1) * 2,
                                 static_cast<cuuint64_t>(Wc) * a.c1 * 2, 32,
                                 static_cast<cuuint64_t>(Hc) * Wc * a.c1 * 2};
        cuuint32_t box[5] = {16, static_cast<cuuint32_t>(kUpW), static_cast<cuuint32_t>(C::kUpRows),
                             1, 1};
        cuuint32_t estr[5] = {1, 1, 1, 1, 1};
        if (enc && enc(&umap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(a.src1),
                       dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
            b.tma_in = 3;
    }
    launch_dependent(conv3x3_kernel<N, RES>, dim3(grid), dim3(kThreads),
                     b.tma_in == 3 ? C::kSmemUp : C::kSmem, stream, b, omap, imap, umap);
    count_launch();
    return launch_status();
}

template <int N>
int launch(const ConvArgs &a, cudaStream_t stream) {
    const int64_t wbytes = static_cast<int64_t>(a.cin_pad / 16) * Cfg<N, false>::kB;
    // N = 192 (data gradients of the 192-channel decoder input) always streams:
    // its weights exceed the resident region at every cin_pad above 16
    if constexpr (N != 192) {
        if (wbytes <= kResidentMax) return launch_variant<N, true>(a, stream);
    }
    return launch_variant<N, false>(a, stream);
}

}  // namespace

int pack_weights(const float *w, int cin, int cout, int transpose, int cin_pad, int n,
                 __nv_bfloat16 *dst, cudaStream_t stream) {
    const int64_t total = static_cast<int64_t>(cin_pad / 16) * 9 * 2 * n * 8;
    if (total == 0) return SPP_OK;
    const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, 4 * sm_count()));
    pack_weights_kernel<<<grid, 256, 0, stream>>>(w, cin, cout, transpose, cin_pad, n, dst);
    count_launch();
    return launch_status();
}

int conv3x3(const ConvArgs &a, cudaStream_t stream) {
    if (a.B < 0 || a.H < 0 || a.W < 0 || a.cin_pad <= 0 || a.cin_pad % 16 || !supported_n(a.n))
        return SPP_ERR_ARG;
    if (!a.wpack || !aligned16(a.wpack)) return SPP_ERR_ALIGN;
    switch (a.n) {
        case 16: return launch<16>(a, stream);
        case 32: return launch<32>(a, stream);
        case 64: return launch<64>(a, stream);
        case 96: return launch<96>(a, stream);
        case 128: return launch<128>(a, stream);
        default: return launch<192>(a, stream);
    }
}

}  // namespace conv
}  // namespace spp
