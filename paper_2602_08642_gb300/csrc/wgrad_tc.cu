// Weight gradient of the 3x3 convolution on the tcgen05 tensor cores:
//   gw[co][ci][dy][dx] = sum over pixels p of g[p][co] * x[p + (dy-1, dx-1)][ci]
//   gb[co]             = sum over pixels p of g[p][co]
// BF16 operands, FP32 accumulation.
//
// GEMM view: M = 9 * cin_pad rows (tap-major, then input channel), N = the
// output channels (padded to 16), K = the pixels.  Grid (M tiles of 128
// rows) x (pixel splits); each CTA accumulates its rows over its share of
// the pixels in TMEM and writes an FP32 partial sum; a second kernel adds
// the partials in a fixed order (the result is deterministic) and writes gw
// and gb in the natural layout.
//
// K chunk: 64 consecutive pixels of one image row.  Both operands must be
// K-major (pixels contiguous inside a core matrix) while the tensors are
// stored pixel-major (NHWC), so each producer thread loads the 8 x 16-byte
// rows of one 8-pixel x 8-channel block (the im2col gather of its tap, with
// the fused pooling / upsample / concatenation of the layer's input), turns
// the 8x8 BF16 block over with byte permutes and stores it as one core
// matrix.  Warp roles, stage recycling and the bounded waits are those of
// conv_tc.cu.
#include <cuda_bf16.h>

#include <algorithm>

#include "conv_src.cuh"
#include "conv_tc.cuh"
#include "spp_internal.cuh"
#include "tc_common.cuh"

namespace spp {
namespace conv {
namespace {

constexpr int kKP = 64;  // pixels per K chunk
constexpr int kThreads = 288;
constexpr int kHeader = 256;
constexpr int kNS = 4;

template <int N>
struct WCfg {
    static constexpr int kA = 128 * kKP * 2;  // 16 KB
    static constexpr int kB = N * kKP * 2;
    static constexpr int kStage = kA + kB;
    static constexpr int kSmem = kHeader + kNS * kStage + 128;
    static constexpr int kCols = tc::pow2_cols(N);
};

struct WBars {
    uint64_t full[kNS];
    uint64_t empty[kNS];
    uint64_t accf;
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

// 8x8 transpose of 16-bit values: in[p] holds channels 0..7 of pixel p,
// out[c] receives pixels 0..7 of channel c.
__device__ __forceinline__ void transpose8x8(const uint4 (&in)[8], uint4 (&out)[8]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint32_t o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t *w0 = &in[2 * q].x, *w1 = &in[2 * q + 1].x;
            o[q] = __byte_perm(w0[c >> 1], w1[c >> 1], (c & 1) ? 0x7632 : 0x5410);
        }
        out[c] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

template <int N>
__global__ void __launch_bounds__(kThreads, 1) wgrad_kernel(const WgradArgs a) {
    using C = WCfg<N>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char *base = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
    WBars &bars = *reinterpret_cast<WBars *>(base);
    unsigned char *stages = base + kHeader;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x, split = blockIdx.y, splits = gridDim.y;
    const int B = a.x.B, H = a.x.H, W = a.x.W;
    const int cw = (W + kKP - 1) / kKP;
    const int64_t nchunks = static_cast<int64_t>(B) * H * cw;
    const int mpad = gridDim.x * 128;

    if (tid == 0) {
        for (int s = 0; s < kNS; ++s) {
            tc::mbar_init(&bars.full[s], 128);
            tc::mbar_init(&bars.empty[s], 1);
        }
        tc::mbar_init(&bars.accf, 1);
        tc::mbar_init(&bars.drain, 1);
        bars.abort = 0;
        tc::fence_mbar_init();
    }
    if (warp == 8) tc::tmem_alloc(&bars.tmem_base, C::kCols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = bars.tmem_base;
    volatile int *abort_flag = &bars.abort;
    auto fail = [&]() {
        *abort_flag = 1;
        set_status(a.status, SPP_ERR_TIMEOUT);
    };

    if (warp >= 4 && warp < 8) {
        // ---------------------------------------------------------- producers
        const int ptid = tid - 128;
        const int ga = ptid >> 3, ja = ptid & 7;  // A block: row group, pixel group
        const int m0 = mt * 128 + ga * 8;
        const int tap = m0 / a.x.cin_pad, ci0 = m0 - tap * a.x.cin_pad;
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        const bool has_b = ptid < N;
        const int gb_ = ptid >> 3, jb = ptid & 7;  // B block: channel group, pixel group
        float bsum[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) bsum[e] = 0.f;
        uint32_t it = 0;
        for (int64_t q = split; q < nchunks; q += splits, ++it) {
            const int s = static_cast<int>(it % kNS);
            const uint32_t ph = (it / kNS) & 1u;
            if (!tc::mbar_wait(&bars.empty[s], ph ^ 1u, abort_flag)) {
                fail();
                break;
            }
            const int b = static_cast<int>(q / (static_cast<int64_t>(H) * cw));
            const int r = static_cast<int>(q - static_cast<int64_t>(b) * H * cw);
            const int y = r / cw, x0 = (r % cw) * kKP;
            unsigned char *As = stages + s * C::kStage;
            unsigned char *Bs = As + C::kA;
            {
                uint4 v[8], t[8];
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    const int x = x0 + 8 * ja + p;
                    v[p] = (tap < 9 && x < W) ? load_chunk(a.x, b, y + dy, x + dx, ci0)
                                              : make_uint4(0, 0, 0, 0);
                }
                transpose8x8(v, t);
                uint4 *dst = reinterpret_cast<uint4 *>(As + ja * 2048 + ga * 128);
#pragma unroll
                for (int c = 0; c < 8; ++c) dst[c] = t[c];
            }
            if (has_b) {
                uint4 v[8], t[8];
#pragma unroll
                for (int p = 0; p < 8; ++p) {
                    const int x = x0 + 8 * jb + p;
                    v[p] = x < W ? load_chunk(a.g, b, y, x, 8 * gb_) : make_uint4(0, 0, 0, 0);
                    const uint32_t *u = &v[p].x;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float2 f = unpack_bf16x2(u[k]);
                        bsum[2 * k] += f.x;
                        bsum[2 * k + 1] += f.y;
                    }
                }
                transpose8x8(v, t);
                uint4 *dst = reinterpret_cast<uint4 *>(Bs + jb * (N * 16) + gb_ * 128);
#pragma unroll
                for (int c = 0; c < 8; ++c) dst[c] = t[c];
            }
            tc::fence_proxy_async();
            tc::mbar_arrive(&bars.full[s]);
        }
        if (has_b && mt == 0) {
            float *pb = a.pbias + (static_cast<int64_t>(split) * 8 + jb) * N + 8 * gb_;
#pragma unroll
            for (int e = 0; e < 8; ++e) pb[e] = bsum[e];
        }
    } else if (warp == 8) {
        // -------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(128, N);
            uint32_t it = 0;
            bool ok = true;
            for (int64_t q = split; q < nchunks; q += splits, ++it) {
                const int s = static_cast<int>(it % kNS);
                if (!tc::mbar_wait(&bars.full[s], (it / kNS) & 1u, abort_flag)) {
                    fail();
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t a_base = tc::smem_u32(stages + s * C::kStage);
                const uint32_t b_base = a_base + C::kA;
#pragma unroll
                for (int ks = 0; ks < kKP / 16; ++ks) {
                    tc::mma_bf16(tmem, tc::smem_desc(a_base + ks * 2 * 2048, 2048, 128),
                                 tc::smem_desc(b_base + ks * 2 * N * 16, N * 16, 128), idesc,
                                 (it | ks) != 0);
                }
                tc::mma_commit(&bars.empty[s]);
            }
            if (ok) {
                tc::mma_commit(&bars.accf);
            } else if (it > 0) {
                tc::mma_commit(&bars.drain);
                (void)tc::mbar_wait(&bars.drain, 0, nullptr);
            }
        }
        __syncwarp();
    } else {
        // ----------------------------------------------------------- epilogue
        const bool any = split < nchunks;
        bool ok = true;
        if (any && !tc::mbar_wait(&bars.accf, 0, abort_flag)) {
            fail();
            ok = false;
        }
        if (ok) {
            tc::tc_fence_after();
            const int m = mt * 128 + warp * 32 + lane;
#pragma unroll 1
            for (int j0 = 0; j0 < N; j0 += 16) {
                uint32_t v[16];
                tc::tmem_ld16(tmem + (static_cast<uint32_t>(warp * 32) << 16) + j0, v);
                tc::tmem_wait_ld();
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    a.partial[(static_cast<int64_t>(split) * N + j0 + e) * mpad + m] =
                        any ? __uint_as_float(v[e]) : 0.f;
            }
        }
    }

    tc::tc_fence_before();
    __syncthreads();
    if (warp == 8) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, C::kCols);
    }
}

// gw[co][ci][ky][kx] = sum_s partial[s][co][tap * cin_pad + ci]; gb[co] =
// sum_s sum_j pbias[s][j][co].  Fixed summation order.
__global__ void wgrad_reduce_kernel(const float *__restrict__ partial,
                                    const float *__restrict__ pbias, int splits, int n, int mpad,
                                    int cin, int cin_pad, int cout, float *__restrict__ gw,
                                    float *__restrict__ gb) {
    const int64_t total = static_cast<int64_t>(cout) * cin * 9;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
         idx < total + cout; idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (idx < total) {
            const int tap = static_cast<int>(idx % 9);
            const int ci = static_cast<int>((idx / 9) % cin);
            const int co = static_cast<int>(idx / (9 * static_cast<int64_t>(cin)));
            const int m = tap * cin_pad + ci;
            float acc = 0.f;
            for (int s = 0; s < splits; ++s)
                acc += partial[(static_cast<int64_t>(s) * n + co) * mpad + m];
            gw[idx] = acc;
        } else {
            const int co = static_cast<int>(idx - total);
            float acc = 0.f;
            for (int s = 0; s < splits; ++s)
                for (int j = 0; j < 8; ++j) acc += pbias[(static_cast<int64_t>(s) * 8 + j) * n + co];
            if (gb) gb[co] = acc;
        }
    }
}

template <int N>
int launch_wgrad(const WgradArgs &a, int mtiles, int splits, cudaStream_t stream) {
    using C = WCfg<N>;
    static int configured_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        if (cudaFuncSetAttribute(wgrad_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 C::kSmem) != cudaSuccess)
            return SPP_ERR_CUDA;
        configured_dev = dev;
    }
    wgrad_kernel<N><<<dim3(mtiles, splits), kThreads, C::kSmem, stream>>>(a);
    count_launch();
    return launch_status();
}

}  // namespace

int wgrad_splits(int B, int W, int H, int cin_pad) {
    const int mtiles = (9 * cin_pad + 127) / 128;
    const int64_t nchunks = static_cast<int64_t>(B) * H * ((W + kKP - 1) / kKP);
    const int want = std::max(1, sm_count() / mtiles);
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(nchunks, want)));
}

size_t wgrad_workspace_bytes(int B, int W, int H, int cin_pad, int n) {
    const int mtiles = (9 * cin_pad + 127) / 128;
    const int splits = wgrad_splits(B, W, H, cin_pad);
    return sizeof(float) * (static_cast<size_t>(splits) * n * mtiles * 128 +
                            static_cast<size_t>(splits) * 8 * n) + 256;
}

int wgrad(const WgradArgs &a0, float *gw, float *gb, void *ws, cudaStream_t stream) {
    WgradArgs a = a0;
    const int B = a.x.B, W = a.x.W, H = a.x.H;
    if (a.n != 32 && a.n != 64 && a.n != 128) return SPP_ERR_ARG;
    if (a.x.cin_pad <= 0 || a.x.cin_pad % 16) return SPP_ERR_ARG;
    const int64_t npix = static_cast<int64_t>(B) * W * H;
    const int mtiles = (9 * a.x.cin_pad + 127) / 128;
    const int splits = wgrad_splits(B, W, H, a.x.cin_pad);
    const int mpad = mtiles * 128;
    a.partial = static_cast<float *>(ws);
    a.pbias = a.partial + static_cast<size_t>(splits) * a.n * mpad;
    if (npix > 0) {
        int rc;
        switch (a.n) {
            case 32: rc = launch_wgrad<32>(a, mtiles, splits, stream); break;
            case 64: rc = launch_wgrad<64>(a, mtiles, splits, stream); break;
            default: rc = launch_wgrad<128>(a, mtiles, splits, stream); break;
        }
        if (rc != SPP_OK) return rc;
    } else {
        if (cudaMemsetAsync(ws, 0, wgrad_workspace_bytes(B, W, H, a.x.cin_pad, a.n), stream) !=
            cudaSuccess)
            return SPP_ERR_CUDA;
    }
    const int64_t total = static_cast<int64_t>(a.cout) * a.cin * 9 + a.cout;
    const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, 4 * sm_count()));
    wgrad_reduce_kernel<<<grid, 256, 0, stream>>>(a.partial, a.pbias, splits, a.n, mpad, a.cin,
                                                  a.x.cin_pad, a.cout, gw, gb);
    count_launch();
    return launch_status();
}

}  // namespace conv
}  // namespace spp
