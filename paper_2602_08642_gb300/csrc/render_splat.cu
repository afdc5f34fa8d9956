// a4: renderer stand-in, and a5: normalised splat (Eq. stoch_rnoisy) with the
// average-pool pyramid (Eq. app-pyramid) of arXiv 2602.08642.
#include "render_common.cuh"
#include "spp_internal.cuh"

namespace spp {
namespace {

constexpr int kRenderThreads = 256;

// Sample t of the list: pixel i = sample_pixel[t], slot k = t - offsets[i];
// value clean_i * render_factor(key, i, k).
__global__ void __launch_bounds__(kRenderThreads)
render_kernel(const float *__restrict__ clean, const int32_t *__restrict__ offsets,
              const int32_t *__restrict__ sample_pixel, const long long *__restrict__ total,
              long long capacity, long long N, uint64_t key, float4 *__restrict__ rgb) {
    pdl_wait();
    pdl_trigger();
    long long T = *total;
    if (T > capacity) T = capacity;
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long t = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; t < T;
         t += stride) {
        const int i = sample_pixel[t];
        if (i < 0 || i >= N) continue;
        const uint64_t k = static_cast<uint64_t>(t - offsets[i]);
        const float g = render_factor(key, static_cast<uint64_t>(i), k);
        rgb[t] = make_float4(clean[i] * g, clean[N + i] * g, clean[2 * N + i] * g, 0.0f);
    }
}

constexpr int kSplatTX = 32;
constexpr int kSplatTY = 8;
constexpr int kSplatRows = 2;                    // rows per thread
constexpr int kSplatH = kSplatTY * kSplatRows;   // 16: covers one level-4 block
constexpr int kMaxLevels = 5;

struct LayerPtrs {
    float *p[kMaxLevels];
};

// One block = 32 x 16 full-resolution pixels.  Each pixel gathers its slots
// (the list is ordered by pixel), normalises by s_i, and the block reduces
// 2x2 means level by level in shared memory.
__global__ void __launch_bounds__(kSplatTX *kSplatTY)
splat_kernel(const int32_t *__restrict__ offsets, const float4 *__restrict__ rgb,
             const float *__restrict__ s, const float *__restrict__ hw, long long capacity, int W,
             int H, int L, LayerPtrs layers) {
    __shared__ float buf[2][3][kSplatH][kSplatTX + 1];
    pdl_wait();
    pdl_trigger();
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * kSplatTX, y0 = blockIdx.y * kSplatH;
    const long long N = static_cast<long long>(W) * H;
    // all independent per-pixel loads of both rows first, then the samples
    long long beg[kSplatRows], end[kSplatRows];
    float wl[kSplatRows], si[kSplatRows];
    bool in[kSplatRows];
#pragma unroll
    for (int r = 0; r < kSplatRows; ++r) {
        const int x = x0 + tx, y = y0 + ty + kSplatTY * r;
        in[r] = x < W && y < H;
        beg[r] = 0;
        end[r] = 0;
        wl[r] = 1.0f;
        si[r] = 1.0f;
        if (in[r]) {
            const long long i = static_cast<long long>(y) * W + x;
            beg[r] = __ldg(offsets + i);
            end[r] = __ldg(offsets + i + 1);
            wl[r] = __ldg(hw + i);
            si[r] = __ldg(s + i);
        }
    }
    float4 first[kSplatRows], last[kSplatRows];
#pragma unroll
    for (int r = 0; r < kSplatRows; ++r) {
        if (beg[r] < 0) beg[r] = 0;
        if (end[r] > capacity) end[r] = capacity;
        first[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        last[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (end[r] > beg[r]) {
            last[r] = __ldcs(rgb + end[r] - 1);                       // the holdout slot
            if (end[r] - beg[r] >= 2) first[r] = __ldcs(rgb + beg[r]);  // the first regular slot
        }
    }
#pragma unroll
    for (int r = 0; r < kSplatRows; ++r) {
        const int ly = ty + kSplatTY * r;
        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
        if (in[r]) {
            const long long i = static_cast<long long>(y0 + ly) * W + x0 + tx;
            if (end[r] > beg[r]) {
                a0 = first[r].x;
                a1 = first[r].y;
                a2 = first[r].z;
                for (long long t = beg[r] + 1; t < end[r] - 1; ++t) {  // slots beyond two
                    const float4 v = __ldcs(rgb + t);
                    a0 += v.x;
                    a1 += v.y;
                    a2 += v.z;
                }
                a0 = __fmaf_rn(wl[r], last[r].x, a0);
                a1 = __fmaf_rn(wl[r], last[r].y, a1);
                a2 = __fmaf_rn(wl[r], last[r].z, a2);
                a0 = __fdiv_rn(a0, si[r]);
                a1 = __fdiv_rn(a1, si[r]);
                a2 = __fdiv_rn(a2, si[r]);
            }
            float *L0 = layers.p[0];
            __stcs(L0 + i, a0);
            __stcs(L0 + N + i, a1);
            __stcs(L0 + 2 * N + i, a2);
        }
        buf[0][0][ly][tx] = a0;
        buf[0][1][ly][tx] = a1;
        buf[0][2][ly][tx] = a2;
    }
    __syncthreads();
    const int tid = ty * kSplatTX + tx;
#pragma unroll
    for (int l = 1; l < kMaxLevels; ++l) {
        if (l >= L) break;
        const int src = (l - 1) & 1, dst = l & 1;
        const int bw = kSplatTX >> l, bh = kSplatH >> l;
        const int Wl = W >> l, Hl = H >> l;
        const long long Nl = static_cast<long long>(Wl) * Hl;
        if (tid < bw * bh) {
            const int cx = tid % bw, cy = tid / bw;
            const int gx = (x0 >> l) + cx, gy = (y0 >> l) + cy;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float v = 0.25f * ((buf[src][c][2 * cy][2 * cx] + buf[src][c][2 * cy][2 * cx + 1]) +
                                         (buf[src][c][2 * cy + 1][2 * cx] +
                                          buf[src][c][2 * cy + 1][2 * cx + 1]));
                buf[dst][c][cy][cx] = v;
                if (gx < Wl && gy < Hl) layers.p[l][c * Nl + static_cast<long long>(gy) * Wl + gx] = v;
            }
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace spp

extern "C" {

int spp_render_synthetic(const float *clean, const int32_t *offsets, const int32_t *sample_pixel,
                         const int64_t *total, int64_t capacity, int W, int H, uint64_t seed,
                         uint32_t frame, float *rgb, cudaStream_t stream) {
    using namespace spp;
    if (W < 0 || H < 0 || capacity < 0) return SPP_ERR_ARG;
    if (!clean || !offsets || !total) return SPP_ERR_ARG;
    if (capacity > 0 && (!sample_pixel || !rgb)) return SPP_ERR_ARG;
    if (!aligned16(clean) || !aligned16(offsets) || !aligned16(total) ||
        (rgb && !aligned16(rgb)) || (sample_pixel && !aligned16(sample_pixel)))
        return SPP_ERR_ALIGN;
    const long long N = static_cast<long long>(W) * H;
    if (N == 0 || capacity == 0) return SPP_OK;
    long long grid = (capacity + kRenderThreads - 1) / kRenderThreads;
    const long long max_grid = static_cast<long long>(sm_count()) * 8;
    if (grid > max_grid) grid = max_grid;
    launch_dependent(render_kernel, dim3(static_cast<unsigned>(grid)), dim3(kRenderThreads), 0,
                     stream, clean, offsets, sample_pixel,
                     reinterpret_cast<const long long *>(total), capacity, N,
                     stream_key(seed, frame), reinterpret_cast<float4 *>(rgb));
    count_launch();
    return launch_status();
}

int spp_splat_samples(const int32_t *offsets, const float *rgb, const float *s,
                      const float *holdout_w, int64_t capacity, int W, int H, int L,
                      float *const *layers, cudaStream_t stream) {
    using namespace spp;
    if (W < 0 || H < 0 || capacity < 0 || !layers) return SPP_ERR_ARG;
    if (L < 1 || L > kMaxLevels) return SPP_ERR_SHAPE;
    if ((W % (1 << (L - 1))) != 0 || (H % (1 << (L - 1))) != 0) return SPP_ERR_SHAPE;
    if (!offsets || !s || !holdout_w || (capacity > 0 && !rgb)) return SPP_ERR_ARG;
    LayerPtrs lp{};
    for (int l = 0; l < L; ++l) {
        if (!layers[l]) return SPP_ERR_ARG;
        if (!aligned16(layers[l])) return SPP_ERR_ALIGN;
        lp.p[l] = layers[l];
    }
    if (!aligned16(offsets) || !aligned16(s) || !aligned16(holdout_w) || (rgb && !aligned16(rgb)))
        return SPP_ERR_ALIGN;
    if (static_cast<long long>(W) * H == 0) return SPP_OK;
    dim3 block(kSplatTX, kSplatTY);
    dim3 grid((W + kSplatTX - 1) / kSplatTX, (H + kSplatH - 1) / kSplatH);
    launch_dependent(splat_kernel, grid, block, 0, stream, offsets,
                     reinterpret_cast<const float4 *>(rgb), s, holdout_w, capacity, W, H, L, lp);
    count_launch();
    return launch_status();
}

}  // extern "C"
