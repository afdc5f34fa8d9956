// The renderer stand-in's sample value (Sec. 3: the renderer traces the
// requested samples; here a unit-mean log-normal factor on the clean image),
// shared by the renderer and by the straight-through estimator's backward,
// which needs the value of a sample the forward did not trace.
#pragma once

#include "spp_internal.cuh"

namespace spp {

// exp(0.8 Z - 0.32) of slot k of pixel i under the stream key of (seed,
// frame): Z from Box-Muller on two 24-bit uniforms of the pixel's SplitMix64
// counters (2k+1, 2k+2).  ln u1 with u1 = (m + 1/2) 2^-24 is taken exactly:
// below 1/2 u1 itself is exact in FP32; above it 1 - u1 = (2(2^24 - m) - 1)
// 2^-25 is, and log1p keeps the steep sqrt(-2 ln u1) near u1 = 1 accurate.
__device__ __forceinline__ float render_factor(uint64_t key, uint64_t i, uint64_t k) {
    const uint64_t hp = stream_bits(key, i);
    const uint64_t b1 = mix64(hp + (2ull * k + 1ull) * kGamma);
    const uint64_t b2 = mix64(hp + (2ull * k + 2ull) * kGamma);
    const uint32_t m1 = static_cast<uint32_t>(b1 >> 40);
    float lnu;
    if (m1 < (1u << 23)) {
        lnu = logf(static_cast<float>(2u * m1 + 1u) * 0x1p-25f);
    } else {
        const uint32_t q = (1u << 24) - m1;
        lnu = log1pf(-static_cast<float>(2u * q - 1u) * 0x1p-25f);
    }
    const float u2 = static_cast<float>(static_cast<uint32_t>(b2 >> 40)) * 0x1p-24f;
    const float z = sqrtf(-2.0f * lnu) * cospif(2.0f * u2);
    return expf(__fmaf_rn(0.8f, z, -0.32f));
}

}  // namespace spp
