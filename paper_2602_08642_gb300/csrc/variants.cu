// Pipeline variants of the ablations of Sec. 7: the low-resolution density
// map.  (The systematic rounding of the sample map lives in alloc.cu, next
// to the stochastic one.)
//
// P d: every f x f block of the density replaced by its mean, summed in FP32
// as a pairwise tree (each row of the block: adjacent pairs, then pairs of
// pairs; then the row sums the same way, top to bottom) and scaled by 1/f^2
// (exact).  P is a symmetric projection, so the same call maps a gradient
// with respect to P d back to d.
#include <algorithm>

#include "spp_internal.cuh"

namespace spp {
namespace {

template <int F>
__device__ __forceinline__ float tree_sum(const float (&v)[F]) {
    float t[F];
#pragma unroll
    for (int k = 0; k < F; ++k) t[k] = v[k];
#pragma unroll
    for (int w = F; w > 1; w >>= 1) {
#pragma unroll
        for (int k = 0; k < w / 2; ++k) t[k] = __fadd_rn(t[2 * k], t[2 * k + 1]);
    }
    return t[0];
}

template <int F>
__global__ void block_mean_kernel(const float *__restrict__ d, int W, int H,
                                  float *__restrict__ out) {
    const int Wc = W / F, Hc = H / F;
    const int64_t n = static_cast<int64_t>(Wc) * Hc;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int xc = static_cast<int>(i % Wc), yc = static_cast<int>(i / Wc);
        float rows[F];
#pragma unroll
        for (int r = 0; r < F; ++r) {
            const float *p = d + static_cast<int64_t>(yc * F + r) * W + xc * F;
            float v[F];
#pragma unroll
            for (int c = 0; c < F; ++c) v[c] = p[c];
            rows[r] = tree_sum<F>(v);
        }
        const float m = __fmul_rn(tree_sum<F>(rows), 1.0f / static_cast<float>(F * F));
#pragma unroll
        for (int r = 0; r < F; ++r) {
            float *o = out + static_cast<int64_t>(yc * F + r) * W + xc * F;
#pragma unroll
            for (int c = 0; c < F; ++c) o[c] = m;
        }
    }
}

}  // namespace
}  // namespace spp

extern "C" int spp_density_lowres(const float *d, int W, int H, int factor, float *out,
                                  cudaStream_t stream) {
    using namespace spp;
    if (!d || !out || W < 0 || H < 0) return SPP_ERR_ARG;
    if (factor != 1 && factor != 2 && factor != 4 && factor != 8) return SPP_ERR_ARG;
    if (W % factor || H % factor) return SPP_ERR_SHAPE;
    if (!aligned16(d) || !aligned16(out)) return SPP_ERR_ALIGN;
    const int64_t n = static_cast<int64_t>(W / factor) * (H / factor);
    if (n == 0) return SPP_OK;
    if (factor == 1) {
        if (d != out &&
            cudaMemcpyAsync(out, d, sizeof(float) * static_cast<size_t>(W) * H,
                            cudaMemcpyDeviceToDevice, stream) != cudaSuccess)
            return SPP_ERR_CUDA;
        return SPP_OK;
    }
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * sm_count())));
    switch (factor) {
        case 2: block_mean_kernel<2><<<grid, 256, 0, stream>>>(d, W, H, out); break;
        case 4: block_mean_kernel<4><<<grid, 256, 0, stream>>>(d, W, H, out); break;
        default: block_mean_kernel<8><<<grid, 256, 0, stream>>>(d, W, H, out); break;
    }
    count_launch();
    return launch_status();
}
