// The two-stage pipeline's per-pixel steps (Sec. 3, Sec. 6.2 "Learned
// Demodulation", Sec. 6.3): warped recurrent latents, the sampler's and the
// denoiser's input features, demodulation of the noisy radiance with the
// pyramid built from it (Eq. app-pyramid), remodulation with the tone map,
// and the backward of these steps.  All of them are streaming kernels over
// planar FP32 images (one thread per pixel, grid-stride loops), bound by
// HBM; the networks themselves run in unet.cu / conv_tc.cu.
#include <cuda_bf16.h>

#include <algorithm>

#include "recon_common.cuh"
#include "spp_internal.cuh"

namespace spp {

ToneArgs tone_args(const spp_tonemap *tm);  // reconstruct.cu
bool tone_ok(const ToneArgs &t);

namespace {

constexpr int kLatent = SPP_LATENT_CHANNELS;
constexpr float kDemodClamp = 8.0f;
constexpr float kInvLn100 = 1.0f / 4.605170185988091f;

int grid_for(int64_t n) {
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * sm_count())));
}

// Bilinear tap positions and weights of W_t at pixel (x, y): the sample
// point (x + mv_x, y + mv_y), pixel centres at integers, clamped to the
// frame (the previous-frame warp of Appendix A).
struct Taps {
    int64_t i00, i01, i10, i11;
    float fx, fy;
};
__device__ __forceinline__ Taps warp_taps(const float *__restrict__ mv, int64_t N, int W, int H,
                                          int x, int y, int64_t i) {
    const float mx = mv[i], my = mv[N + i];
    const float flx = floorf(mx), fly = floorf(my);
    const float ix = fminf(fmaxf(flx, -1048576.0f), 1048576.0f);
    const float iy = fminf(fmaxf(fly, -1048576.0f), 1048576.0f);
    float fx = mx - flx, fy = my - fly;
    int X0 = x + static_cast<int>(ix), Y0 = y + static_cast<int>(iy);
    if (X0 < 0) { X0 = 0; fx = 0.0f; } else if (X0 >= W - 1) { X0 = W - 1; fx = 0.0f; }
    if (Y0 < 0) { Y0 = 0; fy = 0.0f; } else if (Y0 >= H - 1) { Y0 = H - 1; fy = 0.0f; }
    const int X1 = X0 + 1 < W ? X0 + 1 : W - 1;
    const int Y1 = Y0 + 1 < H ? Y0 + 1 : H - 1;
    Taps t;
    t.i00 = static_cast<int64_t>(Y0) * W + X0;
    t.i01 = static_cast<int64_t>(Y0) * W + X1;
    t.i10 = static_cast<int64_t>(Y1) * W + X0;
    t.i11 = static_cast<int64_t>(Y1) * W + X1;
    t.fx = fx;
    t.fy = fy;
    return t;
}

__global__ void warp_latent_kernel(const float *__restrict__ raw, const float *__restrict__ mv,
                                   int W, int H, float *__restrict__ out) {
    const int64_t N = static_cast<int64_t>(W) * H;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % W), y = static_cast<int>(i / W);
        const Taps t = warp_taps(mv, N, W, H, x, y, i);
#pragma unroll
        for (int c = 0; c < kLatent; ++c) {
            const float *p = raw + c * N;
            const float a = tanhf(p[t.i00]), b = tanhf(p[t.i01]);
            const float d = tanhf(p[t.i10]), e = tanhf(p[t.i11]);
            out[c * N + i] = (1.0f - t.fy) * ((1.0f - t.fx) * a + t.fx * b) +
                             t.fy * ((1.0f - t.fx) * d + t.fx * e);
        }
    }
}

// The latents passed on, tanh of the raw planes (each source value once).
__global__ void latent_tanh_kernel(const float *__restrict__ raw, int64_t n,
                                   float *__restrict__ out) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[i] = tanhf(raw[i]);
}

// W_t of C planes (the previous-frame warp of Appendix A on every channel).
// CC > 0 fixes the channel count at compile time, so that the 4 CC tap
// loads of a pixel are all in flight at once; CC = 0 takes C at run time.
template <int CC>
__global__ void warp_channels_kernel(const float *__restrict__ src, int C,
                                     const float *__restrict__ mv, int W, int H,
                                     float *__restrict__ out) {
    const int64_t N = static_cast<int64_t>(W) * H;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < N;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % W), y = static_cast<int>(i / W);
        const Taps t = warp_taps(mv, N, W, H, x, y, i);
        auto warp_one = [&](int c) {
            const float *p = src + c * N;
            out[c * N + i] = (1.0f - t.fy) * ((1.0f - t.fx) * __ldg(p + t.i00) + t.fx * __ldg(p + t.i01)) +
                             t.fy * ((1.0f - t.fx) * __ldg(p + t.i10) + t.fx * __ldg(p + t.i11));
        };
        if constexpr (CC > 0) {
#pragma unroll
            for (int c = 0; c < CC; ++c) warp_one(c);
        } else {
            for (int c = 0; c < C; ++c) warp_one(c);
        }
    }
}

// The sampler's 19 input values of pixel i (FP32).
__device__ __forceinline__ void sampler_values(const float *__restrict__ albedo,
                                               const float *__restrict__ normal,
                                               const float *__restrict__ depth,
                                               const float *__restrict__ mv,
                                               const float *__restrict__ prev,
                                               const float *__restrict__ latent, int64_t n,
                                               int64_t i, float (&v)[32]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[c] = albedo[c * n + i];
        v[3 + c] = normal[c * n + i];
        v[9 + c] = prev ? prev[c * n + i] : 0.f;
    }
    v[6] = logf(depth[i]) * kInvLn100;
    v[7] = mv[i] * 0.125f;
    v[8] = mv[n + i] * 0.125f;
#pragma unroll
    for (int c = 0; c < kLatent; ++c) v[12 + c] = latent ? latent[c * n + i] : 0.f;
#pragma unroll
    for (int c = 12 + kLatent; c < 32; ++c) v[c] = 0.f;
}

// The denoiser's 24 input values of pixel i (FP32).
__device__ __forceinline__ void denoiser_values(const float *__restrict__ L0,
                                                const float *__restrict__ s,
                                                const int32_t *__restrict__ counts,
                                                const float *__restrict__ albedo,
                                                const float *__restrict__ normal,
                                                const float *__restrict__ depth,
                                                const float *__restrict__ mv,
                                                const float *__restrict__ prev,
                                                const float *__restrict__ latent, int64_t n,
                                                int64_t i, float (&v)[32]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[c] = log1pf(L0[c * n + i]);
        v[5 + c] = albedo[c * n + i];
        v[8 + c] = normal[c * n + i];
        v[14 + c] = prev ? log1pf(prev[c * n + i]) : 0.f;
    }
    v[3] = log1pf(s[i]);
    v[4] = log1pf(static_cast<float>(counts[i]));
    v[11] = logf(depth[i]) * kInvLn100;
    v[12] = mv[i] * 0.125f;
    v[13] = mv[n + i] * 0.125f;
#pragma unroll
    for (int c = 0; c < kLatent; ++c) v[17 + c] = latent ? latent[c * n + i] : 0.f;
#pragma unroll
    for (int c = 17 + kLatent; c < 32; ++c) v[c] = 0.f;
}

// FP32 planar [C][H][W] (C = 19 or 24) or the network's BF16 NHWC input
// copy [H][W][32] (rounded to nearest even, padding channels zero).
template <bool DENOISER, bool NHWC>
__global__ void features_kernel(const float *__restrict__ L0, const float *__restrict__ s,
                                const int32_t *__restrict__ counts,
                                const float *__restrict__ albedo, const float *__restrict__ normal,
                                const float *__restrict__ depth, const float *__restrict__ mv,
                                const float *__restrict__ prev, const float *__restrict__ latent,
                                int64_t n, float *__restrict__ out,
                                __nv_bfloat16 *__restrict__ out16) {
    constexpr int C = DENOISER ? 17 + kLatent : 12 + kLatent;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float v[32];
        if (DENOISER)
            denoiser_values(L0, s, counts, albedo, normal, depth, mv, prev, latent, n, i, v);
        else
            sampler_values(albedo, normal, depth, mv, prev, latent, n, i, v);
        if (NHWC) {
            uint32_t w[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
                w[k] = *reinterpret_cast<uint32_t *>(&h);
            }
            uint4 *o = reinterpret_cast<uint4 *>(out16 + i * 32);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                o[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) out[c * n + i] = v[c];
        }
    }
}

__global__ void denoiser_features_backward_kernel(const float *__restrict__ L0,
                                                  const float *__restrict__ s,
                                                  const float *__restrict__ g_in, int64_t n,
                                                  float *__restrict__ g_L0,
                                                  float *__restrict__ g_s) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (g_L0) {
#pragma unroll
            for (int c = 0; c < 3; ++c) g_L0[c * n + i] += g_in[c * n + i] / (1.0f + L0[c * n + i]);
        }
        if (g_s) g_s[i] += g_in[3 * n + i] / (1.0f + s[i]);
    }
}

__device__ __forceinline__ float demod_of(float c) {
    return expf(fminf(fmaxf(c, -kDemodClamp), kDemodClamp));
}

// m = exp(clamp(c)), L0d = L0 / m, Wd = warped / m.
__global__ void demodulate_kernel(const float *__restrict__ L0, const float *__restrict__ c,
                                  const float *__restrict__ warped, int64_t n,
                                  float *__restrict__ m, float *__restrict__ L0d,
                                  float *__restrict__ Wd) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float mk = demod_of(c[k * n + i]);
            m[k * n + i] = mk;
            L0d[k * n + i] = L0[k * n + i] / mk;
            if (warped) Wd[k * n + i] = warped[k * n + i] / mk;
        }
    }
}

// Level l (Wl x Hl) as the 2x2 means of level l - 1 (2 Wl x 2 Hl), 3 planes.
__global__ void pool_level_kernel(const float *__restrict__ fine, int Wl, int Hl,
                                  float *__restrict__ coarse) {
    const int64_t n = static_cast<int64_t>(Wl) * Hl;
    const int64_t nf = 4 * n;
    const int Wf = 2 * Wl;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % Wl), y = static_cast<int>(i / Wl);
        const int64_t f = static_cast<int64_t>(2 * y) * Wf + 2 * x;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float *p = fine + k * nf;
            coarse[k * n + i] = 0.25f * ((p[f] + p[f + 1]) + (p[f + Wf] + p[f + Wf + 1]));
        }
    }
}

__global__ void remodulate_tonemap_kernel(const float *__restrict__ R, const float *__restrict__ m,
                                          int64_t n, ToneArgs tm, float *__restrict__ hdr,
                                          float *__restrict__ ldr) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float o0 = m[i] * R[i], o1 = m[n + i] * R[n + i], o2 = m[2 * n + i] * R[2 * n + i];
        hdr[i] = o0;
        hdr[n + i] = o1;
        hdr[2 * n + i] = o2;
        if (ldr) {
            float r, g, b;
            tone_map(o0, o1, o2, tm, r, g, b);
            ldr[i] = r;
            ldr[n + i] = g;
            ldr[2 * n + i] = b;
        }
    }
}

__global__ void scale_kernel(const float *__restrict__ a, const float *__restrict__ b, int64_t n,
                             float *__restrict__ out) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[i] = a[i] * b[i];
}

__global__ void demodulate_backward_kernel(const float *__restrict__ out_hdr,
                                           const float *__restrict__ g_out,
                                           const float *__restrict__ L0d,
                                           const float *__restrict__ g_L0d,
                                           const float *__restrict__ Wd,
                                           const float *__restrict__ g_Wd,
                                           const float *__restrict__ c,
                                           const float *__restrict__ m, int64_t n,
                                           float *__restrict__ g_L0, float *__restrict__ g_c) {
    const int64_t n3 = 3 * n;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n3;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float gl = g_L0d[i];
        float t = g_out[i] * out_hdr[i] - gl * L0d[i];
        if (Wd) t -= g_Wd[i] * Wd[i];
        g_c[i] = fabsf(c[i]) < kDemodClamp ? t : 0.0f;
        g_L0[i] = gl / m[i];
    }
}

}  // namespace
}  // namespace spp

// ------------------------------------------------------------------ C ABI
using spp::aligned16;
using spp::count_launch;
using spp::grid_for;
using spp::launch_status;

extern "C" int spp_warp_latent(const float *raw, const float *mv, int W, int H, float *out,
                               cudaStream_t stream) {
    if (!raw || !mv || !out || W < 0 || H < 0) return SPP_ERR_ARG;
    if (!aligned16(raw) || !aligned16(mv) || !aligned16(out)) return SPP_ERR_ALIGN;
    const int64_t n = static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    spp::warp_latent_kernel<<<grid_for(n), 256, 0, stream>>>(raw, mv, W, H, out);
    count_launch();
    return launch_status();
}

extern "C" int spp_latent_tanh(const float *raw, int W, int H, float *out, cudaStream_t stream) {
    if (!raw || !out || W < 0 || H < 0) return SPP_ERR_ARG;
    if (!aligned16(raw) || !aligned16(out)) return SPP_ERR_ALIGN;
    const int64_t n = static_cast<int64_t>(spp::kLatent) * W * H;
    if (n == 0) return SPP_OK;
    spp::latent_tanh_kernel<<<grid_for(n), 256, 0, stream>>>(raw, n, out);
    count_launch();
    return launch_status();
}

extern "C" int spp_warp_channels(const float *src, int C, const float *mv, int W, int H,
                                 float *out, cudaStream_t stream) {
    if (!src || !mv || !out || C <= 0 || W < 0 || H < 0) return SPP_ERR_ARG;
    if (!aligned16(src) || !aligned16(mv) || !aligned16(out)) return SPP_ERR_ALIGN;
    const int64_t n = static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    if (C == spp::kLatent)
        spp::warp_channels_kernel<spp::kLatent><<<grid_for(n), 256, 0, stream>>>(src, C, mv, W, H,
                                                                                out);
    else
        spp::warp_channels_kernel<0><<<grid_for(n), 256, 0, stream>>>(src, C, mv, W, H, out);
    count_launch();
    return launch_status();
}

extern "C" int spp_assemble_sampler_features(const float *albedo, const float *normal,
                                             const float *depth, const float *mv,
                                             const float *warped_prev_ldr,
                                             const float *warped_latent, int W, int H,
                                             float *in19, cudaStream_t stream) {
    if (W < 0 || H < 0 || !albedo || !normal || !depth || !mv || !in19) return SPP_ERR_ARG;
    if (!aligned16(albedo) || !aligned16(normal) || !aligned16(depth) || !aligned16(mv) ||
        !aligned16(in19) || (warped_prev_ldr && !aligned16(warped_prev_ldr)) ||
        (warped_latent && !aligned16(warped_latent)))
        return SPP_ERR_ALIGN;
    const int64_t n = static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    spp::features_kernel<false, false><<<grid_for(n), 256, 0, stream>>>(
        nullptr, nullptr, nullptr, albedo, normal, depth, mv, warped_prev_ldr, warped_latent, n,
        in19, nullptr);
    count_launch();
    return launch_status();
}

extern "C" int spp_assemble_denoiser_features(const float *L0, const float *s,
                                              const int32_t *counts, const float *albedo,
                                              const float *normal, const float *depth,
                                              const float *mv, const float *warped_prev_hdr,
                                              const float *warped_latent, int W, int H,
                                              float *in24, cudaStream_t stream) {
    if (W < 0 || H < 0 || !L0 || !s || !counts || !albedo || !normal || !depth || !mv || !in24)
        return SPP_ERR_ARG;
    if (!aligned16(L0) || !aligned16(s) || !aligned16(counts) || !aligned16(albedo) ||
        !aligned16(normal) || !aligned16(depth) || !aligned16(mv) || !aligned16(in24) ||
        (warped_prev_hdr && !aligned16(warped_prev_hdr)) ||
        (warped_latent && !aligned16(warped_latent)))
        return SPP_ERR_ALIGN;
    const int64_t n = static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    spp::features_kernel<true, false><<<grid_for(n), 256, 0, stream>>>(
        L0, s, counts, albedo, normal, depth, mv, warped_prev_hdr, warped_latent, n, in24,
        nullptr);
    count_launch();
    return launch_status();
}

extern "C" int spp_assemble_sampler_input(const float *albedo, const float *normal,
                                          const float *depth, const float *mv,
                                          const float *warped_prev_ldr,
                                          const float *warped_latent, int W, int H,
                                          uint16_t *x_nhwc32, cudaStream_t stream) {
    if (W < 0 || H < 0 || !albedo || !normal || !depth || !mv || !x_nhwc32) return SPP_ERR_ARG;
    if (!aligned16(albedo) || !aligned16(normal) || !aligned16(depth) || !aligned16(mv) ||
        !aligned16(x_nhwc32) || (warped_prev_ldr && !aligned16(warped_prev_ldr)) ||
        (warped_latent && !aligned16(warped_latent)))
        return SPP_ERR_ALIGN;
    const int64_t n = static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    spp::features_kernel<false, true><<<grid_for(n), 256, 0, stream>>>(
        nullptr, nullptr, nullptr, albedo, normal, depth, mv, warped_prev_ldr, warped_latent, n,
        nullptr, reinterpret_cast<__nv_bfloat16 *>(x_nhwc32));
    count_launch();
    return launch_status();
}

extern "C" int spp_assemble_denoiser_input(const float *L0, const float *s, const int32_t *counts,
                                           const float *albedo, const float *normal,
                                           const float *depth, const float *mv,
                                           const float *warped_prev_hdr,
                                           const float *warped_latent, int W, int H,
                                           uint16_t *x_nhwc32, cudaStream_t stream) {
    if (W < 0 || H < 0 || !L0 || !s || !counts || !albedo || !normal || !depth || !mv ||
        !x_nhwc32)
        return SPP_ERR_ARG;
    if (!aligned16(L0) || !aligned16(s) || !aligned16(counts) || !aligned16(albedo) ||
        !aligned16(normal) || !aligned16(depth) || !aligned16(mv) || !aligned16(x_nhwc32) ||
        (warped_prev_hdr && !aligned16(warped_prev_hdr)) ||
        (warped_latent && !aligned16(warped_latent)))
        return SPP_ERR_ALIGN;
    const int64_t n = static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    spp::features_kernel<true, true><<<grid_for(n), 256, 0, stream>>>(
        L0, s, counts, albedo, normal, depth, mv, warped_prev_hdr, warped_latent, n, nullptr,
        reinterpret_cast<__nv_bfloat16 *>(x_nhwc32));
    count_launch();
    return launch_status();
}

extern "C" int spp_denoiser_features_backward(const float *L0, const float *s,
                                              const float *grad_in24, int W, int H,
                                              float *grad_L0, float *grad_s,
                                              cudaStream_t stream) {
    if (W < 0 || H < 0 || !L0 || !s || !grad_in24 || (!grad_L0 && !grad_s)) return SPP_ERR_ARG;
    if (!aligned16(L0) || !aligned16(s) || !aligned16(grad_in24) ||
        (grad_L0 && !aligned16(grad_L0)) || (grad_s && !aligned16(grad_s)))
        return SPP_ERR_ALIGN;
    const int64_t n = static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    spp::denoiser_features_backward_kernel<<<grid_for(n), 256, 0, stream>>>(L0, s, grad_in24, n,
                                                                            grad_L0, grad_s);
    count_launch();
    return launch_status();
}

extern "C" int spp_demodulate(const float *L0, const float *c, const float *warped, int W, int H,
                              int L, float *m, float *const *layers, float *warped_out,
                              cudaStream_t stream) {
    if (!L0 || !c || !m || !layers || W < 0 || H < 0 || L < 1 || L > 5) return SPP_ERR_ARG;
    if (warped && !warped_out) return SPP_ERR_ARG;
    for (int l = 0; l < L; ++l)
        if (!layers[l]) return SPP_ERR_ARG;
    if (W % (1 << (L - 1)) || H % (1 << (L - 1))) return SPP_ERR_SHAPE;
    if (!aligned16(L0) || !aligned16(c) || !aligned16(m) || (warped && !aligned16(warped)) ||
        (warped_out && !aligned16(warped_out)))
        return SPP_ERR_ALIGN;
    for (int l = 0; l < L; ++l)
        if (!aligned16(layers[l])) return SPP_ERR_ALIGN;
    const int64_t n = static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    spp::demodulate_kernel<<<grid_for(n), 256, 0, stream>>>(L0, c, warped, n, m, layers[0],
                                                            warped ? warped_out : nullptr);
    count_launch();
    for (int l = 1; l < L; ++l) {
        const int Wl = W >> l, Hl = H >> l;
        spp::pool_level_kernel<<<grid_for(static_cast<int64_t>(Wl) * Hl), 256, 0, stream>>>(
            layers[l - 1], Wl, Hl, layers[l]);
        count_launch();
    }
    return launch_status();
}

extern "C" int spp_remodulate_tonemap(const float *R, const float *m, int W, int H,
                                      const spp_tonemap *tm, float *out_hdr, float *out_ldr,
                                      cudaStream_t stream) {
    if (!R || !m || !out_hdr || W < 0 || H < 0) return SPP_ERR_ARG;
    if (!aligned16(R) || !aligned16(m) || !aligned16(out_hdr) || (out_ldr && !aligned16(out_ldr)))
        return SPP_ERR_ALIGN;
    const spp::ToneArgs t = spp::tone_args(tm);
    if (!spp::tone_ok(t)) return SPP_ERR_ARG;
    const int64_t n = static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    spp::remodulate_tonemap_kernel<<<grid_for(n), 256, 0, stream>>>(R, m, n, t, out_hdr, out_ldr);
    count_launch();
    return launch_status();
}

extern "C" int spp_remodulate_backward(const float *grad_out, const float *m, int W, int H,
                                       float *grad_R, cudaStream_t stream) {
    if (!grad_out || !m || !grad_R || W < 0 || H < 0) return SPP_ERR_ARG;
    if (!aligned16(grad_out) || !aligned16(m) || !aligned16(grad_R)) return SPP_ERR_ALIGN;
    const int64_t n = 3 * static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    spp::scale_kernel<<<grid_for(n), 256, 0, stream>>>(grad_out, m, n, grad_R);
    count_launch();
    return launch_status();
}

extern "C" int spp_demodulate_backward(const float *out_hdr, const float *grad_out,
                                       const float *L0d, const float *grad_L0d, const float *Wd,
                                       const float *grad_Wd, const float *c, const float *m,
                                       int W, int H, float *grad_L0, float *grad_c,
                                       cudaStream_t stream) {
    if (!out_hdr || !grad_out || !L0d || !grad_L0d || !c || !m || !grad_L0 || !grad_c || W < 0 ||
        H < 0 || (Wd && !grad_Wd))
        return SPP_ERR_ARG;
    if (!aligned16(out_hdr) || !aligned16(grad_out) || !aligned16(L0d) || !aligned16(grad_L0d) ||
        !aligned16(c) || !aligned16(m) || !aligned16(grad_L0) || !aligned16(grad_c) ||
        (Wd && (!aligned16(Wd) || !aligned16(grad_Wd))))
        return SPP_ERR_ALIGN;
    const int64_t n = static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    spp::demodulate_backward_kernel<<<grid_for(3 * n), 256, 0, stream>>>(
        out_hdr, grad_out, L0d, grad_L0d, Wd, Wd ? grad_Wd : nullptr, c, m, n, grad_L0, grad_c);
    count_launch();
    return launch_status();
}
