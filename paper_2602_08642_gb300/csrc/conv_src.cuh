// Device-side loaders of the convolution operands shared by the forward /
// data-gradient kernel (conv_tc.cu) and the weight-gradient kernel
// (wgrad_tc.cu): 8 consecutive channels of one pixel of the conceptual
// input tensor, as one 16-byte BF16 chunk, with zero padding outside the
// image and the fused pooling / upsample + concatenation / FP32 conversion
// of the source modes.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "conv_tc.cuh"

namespace spp {
namespace conv {

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ float2 unpack_bf16x2(uint32_t u) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&u);
    return __bfloat1622float2(h);
}

__device__ __forceinline__ uint4 ldg16(const __nv_bfloat16 *p) {
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

// 8 input channels [ch, ch+8) of pixel (b, y, x) of the conceptual input.
__device__ __forceinline__ uint4 load_chunk(const ConvArgs &a, int b, int y, int x, int ch) {
    const uint4 zero = make_uint4(0, 0, 0, 0);
    if (y < 0 || y >= a.H || x < 0 || x >= a.W) return zero;
    switch (a.src_mode) {
        case kSrcNHWC:
            if (ch >= a.c0) return zero;
            return ldg16(a.src0 + ((static_cast<size_t>(b) * a.H + y) * a.W + x) * a.c0 + ch);
        case kSrcPool: {
            if (ch >= a.c0) return zero;
            const int Wf = 2 * a.W;
            const __nv_bfloat16 *p =
                a.src0 + ((static_cast<size_t>(b) * 2 * a.H + 2 * y) * Wf + 2 * x) * a.c0 + ch;
            const uint4 q0 = ldg16(p), q1 = ldg16(p + a.c0);
            const uint4 q2 = ldg16(p + static_cast<size_t>(Wf) * a.c0);
            const uint4 q3 = ldg16(p + static_cast<size_t>(Wf) * a.c0 + a.c0);
            const uint32_t *u0 = &q0.x, *u1 = &q1.x, *u2 = &q2.x, *u3 = &q3.x;
            uint4 r;
            uint32_t *ro = &r.x;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f0 = unpack_bf16x2(u0[k]), f1 = unpack_bf16x2(u1[k]);
                const float2 f2 = unpack_bf16x2(u2[k]), f3 = unpack_bf16x2(u3[k]);
                ro[k] = pack_bf16x2(((f0.x + f1.x) + (f2.x + f3.x)) * 0.25f,
                                    ((f0.y + f1.y) + (f2.y + f3.y)) * 0.25f);
            }
            return r;
        }
        case kSrcConcatUp:
            if (ch < a.c0)
                return ldg16(a.src0 + ((static_cast<size_t>(b) * a.H + y) * a.W + x) * a.c0 + ch);
            if (ch - a.c0 >= a.c1) return zero;
            return ldg16(a.src1 +
                         ((static_cast<size_t>(b) * (a.H >> 1) + (y >> 1)) * (a.W >> 1) + (x >> 1)) *
                             a.c1 +
                         (ch - a.c0));
        default: {  // kSrcPlanarF32
            const size_t plane = static_cast<size_t>(a.H) * a.W;
            const float *p = a.srcf + (static_cast<size_t>(b) * a.cf + ch) * plane +
                             static_cast<size_t>(y) * a.W + x;
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = (ch + e < a.cf) ? __ldg(p + e * plane) : 0.f;
            return make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]),
                              pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
        }
    }
}


// Global address of the 8-channel chunk [ch, ch+8) of pixel (b, y, x) for
// the sources that need no arithmetic (NHWC, upsample + concatenation), or
// nullptr where the chunk is zero padding.
__device__ __forceinline__ const __nv_bfloat16 *chunk_address(const ConvArgs &a, int b, int y,
                                                              int x, int ch) {
    if (y < 0 || y >= a.H || x < 0 || x >= a.W) return nullptr;
    if (ch < a.c0) return a.src0 + ((static_cast<size_t>(b) * a.H + y) * a.W + x) * a.c0 + ch;
    if (a.src_mode != kSrcConcatUp || ch - a.c0 >= a.c1) return nullptr;
    return a.src1 + ((static_cast<size_t>(b) * (a.H >> 1) + (y >> 1)) * (a.W >> 1) + (x >> 1)) * a.c1 +
           (ch - a.c0);
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros
// (and reads nothing).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

}  // namespace conv
}  // namespace spp
