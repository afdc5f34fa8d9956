// Pieces shared by the two reconstruction paths (direct and TMA-pipelined).
#pragma once

#include "spp_internal.cuh"

namespace spp {

struct ToneArgs {
    float alpha, beta, k, s, h;
    float inv_s, inv_h;  // 1/s and 1/h, computed once on the host
};

constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// 2^x on the SFU (relative error about 2^-22; results below 2^-126 flush to
// 0, which only drops softmax weights smaller than 1e-38 of the largest).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x on the SFU (about 1 ulp), for the softmax normalisation.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// tau of Sec. 5: exponential toe below s-1, linear middle, exponential
// shoulder above 1-h.
// Branch-free: one exponential serves whichever tail the argument is in.
// The tails divide by s and by h, uniform over the frame: multiplying by the
// host-computed reciprocals costs one rounding more than a division
// (relative 2^-24), far inside the output tolerance.
__device__ __forceinline__ float tau_curve(float x, float s, float h, float inv_s, float inv_h) {
    const bool toe = x < s - 1.0f;
    const bool mid = !toe && x < 1.0f - h;
    const float arg = toe ? (x + 1.0f - s) * inv_s : -(x + h - 1.0f) * inv_h;
    const float ex = __expf(fminf(arg, 0.0f));
    const float tail = toe ? 0.5f * s * ex : 1.0f - 0.5f * h * ex;
    return mid ? 0.5f * (1.0f + x) : tail;
}

// IEC 61966-2-1 sRGB encoding (branch-free select).
__device__ __forceinline__ float srgb(float v) {
    const float hi = 1.055f * __powf(fmaxf(v, 0.0031308f), 1.0f / 2.4f) - 0.055f;
    return v <= 0.0031308f ? 12.92f * v : hi;
}

// Sec. 5: x_c = alpha (mean + beta (ln L_c - mean) + k), then tau and sRGB.
__device__ __forceinline__ void tone_map(float o0, float o1, float o2, const ToneArgs &tm,
                                         float &r, float &g, float &b) {
    const float l0 = __logf(fmaxf(o0, 0x1p-24f));
    const float l1 = __logf(fmaxf(o1, 0x1p-24f));
    const float l2 = __logf(fmaxf(o2, 0x1p-24f));
    const float mean = (l0 + l1 + l2) * (1.0f / 3.0f);
    r = srgb(tau_curve(tm.alpha * (mean + tm.beta * (l0 - mean) + tm.k), tm.s, tm.h, tm.inv_s,
                       tm.inv_h));
    g = srgb(tau_curve(tm.alpha * (mean + tm.beta * (l1 - mean) + tm.k), tm.s, tm.h, tm.inv_s,
                       tm.inv_h));
    b = srgb(tau_curve(tm.alpha * (mean + tm.beta * (l2 - mean) + tm.k), tm.s, tm.h, tm.inv_s,
                       tm.inv_h));
}

// Launches the TMA-pipelined reconstruction of one level when the level's
// shape allows it (row pitch a multiple of 16 bytes).  Returns false, with
// nothing launched, when it does not; *rc then stays SPP_OK.  warped is
// W_t L_{t-1} at full resolution, or NULL for no temporal term.
bool launch_recon_tma(const float *noisy, const float *logits, int C_total, int C_used,
                      const float *coarse, const float *warped, const uint8_t *mask, int Wl,
                      int Hl, float *out, float *out_ldr, const ToneArgs &tm, int32_t *status,
                      cudaStream_t stream, int *rc);

// Launches the bilinear reprojection W_t L_{t-1} of the previous HDR output.
void launch_warp_prev(const float *prev, const float *mv, int Wl, int Hl, float *warped,
                      cudaStream_t stream);

}  // namespace spp
