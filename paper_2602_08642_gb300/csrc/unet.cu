// The learned predictor (Sec. 3, Sec. 6.3): a U-Net of 3x3 convolutions on
// the tensor cores (conv_tc.cu) that maps the G-buffer features and the
// previous output to the density logit and the kernel logits of the three
// pyramid levels.  This file holds the layer table, parameter packing, the
// feature assembly, the density softmax and the forward orchestration.
#include <cuda_bf16.h>

#include <algorithm>

#include "conv_tc.cuh"
#include "spp_internal.cuh"
#include "unet_internal.cuh"

namespace spp {
namespace unet {

const NetSpec kNets[kNumNets] = {
    {12, {55, 29, 25}},  // joint predictor
    {19, {1, 0, 0}},     // sampler
    {24, {64, 29, 25}},  // denoiser
};

Layer layer(int net, int i) {
    static const Layer trunk[kNumLayers] = {
        {0, 32, 1},    {32, 32, 1}, {32, 64, 1}, {64, 64, 1}, {64, 128, 1},
        {128, 128, 1}, {128, 0, 0}, {192, 64, 1}, {64, 64, 1}, {64, 0, 0},
        {96, 32, 1},   {32, 32, 1}, {32, 0, 0},
    };
    Layer l = trunk[i];
    const NetSpec &n = kNets[net];
    if (i == E0A) l.cin = n.cin;
    if (i == H0) l.cout = n.heads[0];
    if (i == H1) l.cout = n.heads[1];
    if (i == H2) l.cout = n.heads[2];
    return l;
}

int level_of(int i) {
    return (i == E1A || i == E1B || i == D1A || i == D1B || i == H1) ? 1
           : (i == E2A || i == E2B || i == H2)                       ? 2
                                                                     : 0;
}

int round16(int c) { return (c + 15) / 16 * 16; }

int input_channels_padded(int net) { return round16(kNets[net].cin); }

// MMA width of a layer's forward convolution (its output channels, padded).
int fwd_n(int net, int i) {
    const Layer l = layer(net, i);
    return l.relu ? l.cout : (l.cout <= 32 ? 32 : 64);
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

PackedLayout packed_layout(int net, int with_backward) {
    PackedLayout L{};
    size_t off = 0;
    int64_t toff = 0;
    for (int i = 0; i < kNumLayers; ++i) {
        const Layer l = layer(net, i);
        if (l.cout == 0) {
            L.theta_w[i] = L.theta_b[i] = toff;
            L.fwd[i] = L.bias[i] = 0;
            continue;
        }
        L.theta_w[i] = toff;
        L.theta_b[i] = toff + static_cast<int64_t>(l.cout) * l.cin * 9;
        toff = L.theta_b[i] + l.cout;
        L.fwd[i] = off;
        off = align256(off + conv::packed_bytes(round16(l.cin), fwd_n(net, i)));
        L.bias[i] = off;
        off = align256(off + sizeof(float) * fwd_n(net, i));
    }
    L.param_count = toff;
    for (int i = 0; i < kNumLayers; ++i) {
        const Layer l = layer(net, i);
        L.bwd[i] = 0;
        if (with_backward && l.cout > 0) {
            // data-gradient operand: input channels = this layer's outputs,
            // MMA width = its inputs (the input layer's padded to 16 / 32)
            L.bwd[i] = off;
            off = align256(off + conv::packed_bytes(round16(l.cout),
                                                    i == E0A ? round16(l.cin) : l.cin));
        }
    }
    L.total = off;
    return L;
}

ActLayout act_layout(int net, int B, int W, int H) {
    ActLayout A{};
    const size_t p0 = static_cast<size_t>(B) * H * W, p1 = p0 / 4, p2 = p0 / 16;
    size_t off = 0;
    auto take = [&](size_t elems) {
        const size_t o = off;
        off = align256(off + elems * sizeof(__nv_bfloat16));
        return o;
    };
    A.xin_c = input_channels_padded(net);
    A.xin = take(p0 * A.xin_c);
    A.e0a = take(p0 * 32);
    A.s0 = take(p0 * 32);
    A.p0 = take(p1 * 32);
    A.e1a = take(p1 * 64);
    A.s1 = take(p1 * 64);
    A.p1 = take(p2 * 64);
    A.e2a = take(p2 * 128);
    A.bt = take(p2 * 128);
    A.d1a = take(p1 * 64);
    A.t1 = take(p1 * 64);
    A.d0a = take(p0 * 32);
    A.t0 = take(p0 * 32);
    A.zmax = off;
    off = align256(off + sizeof(uint32_t) * std::max(B, 1));
    A.total = off;
    return A;
}

namespace {

__global__ void assemble_kernel(const float *__restrict__ albedo, const float *__restrict__ normal,
                                const float *__restrict__ depth, const float *__restrict__ mv,
                                const float *__restrict__ prev, int64_t n, float *__restrict__ out) {
    const float inv_ln100 = 1.0f / 4.605170185988091f;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        out[i] = albedo[i];
        out[n + i] = albedo[n + i];
        out[2 * n + i] = albedo[2 * n + i];
        out[3 * n + i] = normal[i];
        out[4 * n + i] = normal[n + i];
        out[5 * n + i] = normal[2 * n + i];
        out[6 * n + i] = logf(depth[i]) * inv_ln100;
        out[7 * n + i] = mv[i] * 0.125f;
        out[8 * n + i] = mv[n + i] * 0.125f;
        out[9 * n + i] = prev ? prev[i] : 0.f;
        out[10 * n + i] = prev ? prev[n + i] : 0.f;
        out[11 * n + i] = prev ? prev[2 * n + i] : 0.f;
    }
}

// in12 [B][12][H][W] FP32 -> BF16 [B][H][W][16] (round to nearest even,
// channels 12..15 zero): the layout the first convolution streams.
__global__ void features_nhwc16_kernel(const float *__restrict__ in12, int64_t n, int64_t hw,
                                       __nv_bfloat16 *__restrict__ out) {
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t b = p / hw, i = p - b * hw;
        const float *src = in12 + b * 12 * hw + i;
        uint32_t w[8];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            __nv_bfloat162 h = __floats2bfloat162_rn(__ldg(src + (2 * k) * hw),
                                                     __ldg(src + (2 * k + 1) * hw));
            w[k] = *reinterpret_cast<uint32_t *>(&h);
        }
        w[6] = w[7] = 0;
        uint4 *o = reinterpret_cast<uint4 *>(out + p * 16);
        o[0] = make_uint4(w[0], w[1], w[2], w[3]);
        o[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
}

// in [B][C][H][W] FP32 -> BF16 [B][H][W][CP] (CP = 32; channels C..CP-1 zero).
__global__ void features_nhwc32_kernel(const float *__restrict__ in, int C, int64_t n, int64_t hw,
                                       __nv_bfloat16 *__restrict__ out) {
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t b = p / hw, i = p - b * hw;
        const float *src = in + b * C * hw + i;
        uint32_t w[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float lo = 2 * k < C ? __ldg(src + (2 * k) * hw) : 0.f;
            const float hi = 2 * k + 1 < C ? __ldg(src + (2 * k + 1) * hw) : 0.f;
            __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
            w[k] = *reinterpret_cast<uint32_t *>(&h);
        }
        uint4 *o = reinterpret_cast<uint4 *>(out + p * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    }
}

__global__ void copy_bias_kernel(const float *__restrict__ b, int cout, int n, float *__restrict__ dst) {
    const int i = threadIdx.x;
    if (i < n) dst[i] = i < cout ? b[i] : 0.f;
}

// Order-preserving map of a float to an unsigned integer (for atomicMax).
__device__ __forceinline__ uint32_t ordered(float f) {
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unordered(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// zmax[b] = max over the frame of z[b * stride + i]
__global__ void zmax_kernel(const float *__restrict__ zplane, int64_t hw, int64_t stride,
                            uint32_t *__restrict__ zmax) {
    const int b = blockIdx.y;
    const float *z = zplane + static_cast<int64_t>(b) * stride;
    float m = -INFINITY;
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < hw;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        m = fmaxf(m, z[i]);
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? wm[threadIdx.x] : -INFINITY;
#pragma unroll
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) atomicMax(zmax + b, ordered(m));
    }
}

__global__ void density_kernel(const float *__restrict__ zplane, int64_t hw, int64_t stride,
                               const uint32_t *__restrict__ zmax, float *__restrict__ d) {
    const int b = blockIdx.y;
    const float *z = zplane + static_cast<int64_t>(b) * stride;
    const float m = unordered(zmax[b]);
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < hw;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        d[static_cast<int64_t>(b) * hw + i] = expf(z[i] - m);
}

}  // namespace

conv::ConvArgs layer_input(int net, int i, int B, int W, int H, const unsigned char *ws) {
    const ActLayout A = act_layout(net, B, W, H);
    auto act = [&](size_t off) { return reinterpret_cast<const __nv_bfloat16 *>(ws + off); };
    conv::ConvArgs a;
    const int level = level_of(i);
    a.B = B;
    a.W = W >> level;
    a.H = H >> level;
    a.cin_pad = i == E0A ? A.xin_c : round16(layer(net, i).cin);
    a.src_mode = conv::kSrcNHWC;
    switch (i) {
        case E0A: a.src0 = act(A.xin); a.c0 = A.xin_c; break;
        case E0B: a.src0 = act(A.e0a); a.c0 = 32; break;
        case E1A: a.src0 = act(A.p0); a.c0 = 32; break;
        case E1B: a.src0 = act(A.e1a); a.c0 = 64; break;
        case E2A: a.src0 = act(A.p1); a.c0 = 64; break;
        case E2B: a.src0 = act(A.e2a); a.c0 = 128; break;
        case H2: a.src0 = act(A.bt); a.c0 = 128; break;
        case D1A:
            a.src_mode = conv::kSrcConcatUp;
            a.src0 = act(A.s1); a.c0 = 64; a.src1 = act(A.bt); a.c1 = 128;
            break;
        case D1B: a.src0 = act(A.d1a); a.c0 = 64; break;
        case H1: a.src0 = act(A.t1); a.c0 = 64; break;
        case D0A:
            a.src_mode = conv::kSrcConcatUp;
            a.src0 = act(A.s0); a.c0 = 32; a.src1 = act(A.t1); a.c1 = 64;
            break;
        case D0B: a.src0 = act(A.d0a); a.c0 = 32; break;
        default: a.src0 = act(A.t0); a.c0 = 32; break;  // H0
    }
    return a;
}

size_t layer_output(int i, const ActLayout &A) {
    static const int idx[kNumLayers] = {0, 1, 2, 3, 4, 5, -1, 6, 7, -1, 8, 9, -1};
    const size_t offs[10] = {A.e0a, A.s0, A.e1a, A.s1, A.e2a, A.bt, A.d1a, A.t1, A.d0a, A.t0};
    return idx[i] < 0 ? static_cast<size_t>(-1) : offs[idx[i]];
}

int density_softmax(const float *z, int B, int64_t hw, int64_t batch_stride, float *d,
                    uint32_t *zmax, cudaStream_t stream) {
    if (cudaMemsetAsync(zmax, 0, sizeof(uint32_t) * B, stream) != cudaSuccess) return SPP_ERR_CUDA;
    const int gx = static_cast<int>(std::min<int64_t>((hw + 255) / 256, 2 * sm_count()));
    zmax_kernel<<<dim3(gx, B), 256, 0, stream>>>(z, hw, batch_stride, zmax);
    density_kernel<<<dim3(gx, B), 256, 0, stream>>>(z, hw, batch_stride, zmax, d);
    count_launch(2);
    return launch_status();
}

int forward(int net, const unsigned char *packed, const float *in, int B, int W, int H,
            float *density, float *head0, float *head1, float *head2, unsigned char *ws,
            int32_t *status, cudaStream_t stream) {
    const PackedLayout P = packed_layout(net, 0);
    const ActLayout A = act_layout(net, B, W, H);
    float *heads[kNumLayers] = {};
    heads[H0] = head0;
    heads[H1] = head1;
    heads[H2] = head2;
    if (in) {  // else the BF16 NHWC input copy is already in the workspace
        const int64_t n = static_cast<int64_t>(B) * W * H;
        const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 8 * sm_count()));
        auto *x = reinterpret_cast<__nv_bfloat16 *>(ws + A.xin);
        if (A.xin_c == 16)
            features_nhwc16_kernel<<<grid, 256, 0, stream>>>(in, n, static_cast<int64_t>(W) * H, x);
        else
            features_nhwc32_kernel<<<grid, 256, 0, stream>>>(in, kNets[net].cin, n,
                                                             static_cast<int64_t>(W) * H, x);
        count_launch();
        if (launch_status() != SPP_OK) return SPP_ERR_CUDA;
    }
    static const int order[kNumLayers] = {E0A, E0B, E1A, E1B, E2A, E2B, H2,
                                          D1A, D1B, H1,  D0A, D0B, H0};
    for (int k = 0; k < kNumLayers; ++k) {
        const int i = order[k];
        const Layer l = layer(net, i);
        if (l.cout == 0) continue;
        conv::ConvArgs a = layer_input(net, i, B, W, H, ws);
        a.n = fwd_n(net, i);
        a.cout = l.cout;
        a.wpack = reinterpret_cast<const __nv_bfloat16 *>(packed + P.fwd[i]);
        a.bias = reinterpret_cast<const float *>(packed + P.bias[i]);
        a.status = status;
        if (l.relu) {
            a.epi_mode = conv::kEpiReluBF16;
            a.out = reinterpret_cast<__nv_bfloat16 *>(ws + layer_output(i, A));
            if (i == E0B) a.pool_out = reinterpret_cast<__nv_bfloat16 *>(ws + A.p0);
            if (i == E1B) a.pool_out = reinterpret_cast<__nv_bfloat16 *>(ws + A.p1);
        } else {
            a.epi_mode = conv::kEpiF32Planar;
            a.outf = heads[i];
        }
        const int rc = conv::conv3x3(a, stream);
        if (rc != SPP_OK) return rc;
    }
    if (net == kNetJoint && density) {
        const int64_t hw = static_cast<int64_t>(W) * H;
        return density_softmax(head0 + kDensityChannel * hw, B, hw, 55 * hw, density,
                               reinterpret_cast<uint32_t *>(ws + A.zmax), stream);
    }
    return launch_status();
}

int pack(int net, const float *theta, int with_backward, unsigned char *packed,
         cudaStream_t stream) {
    const PackedLayout P = packed_layout(net, with_backward);
    for (int i = 0; i < kNumLayers; ++i) {
        const Layer l = layer(net, i);
        if (l.cout == 0) continue;
        int rc = conv::pack_weights(theta + P.theta_w[i], l.cin, l.cout, 0, round16(l.cin),
                                    fwd_n(net, i),
                                    reinterpret_cast<__nv_bfloat16 *>(packed + P.fwd[i]), stream);
        if (rc != SPP_OK) return rc;
        copy_bias_kernel<<<1, 256, 0, stream>>>(theta + P.theta_b[i], l.cout, fwd_n(net, i),
                                                reinterpret_cast<float *>(packed + P.bias[i]));
        count_launch();
        if (with_backward) {
            rc = conv::pack_weights(theta + P.theta_w[i], l.cin, l.cout, 1, round16(l.cout),
                                    i == E0A ? round16(l.cin) : l.cin,
                                    reinterpret_cast<__nv_bfloat16 *>(packed + P.bwd[i]), stream);
            if (rc != SPP_OK) return rc;
        }
    }
    return launch_status();
}

int assemble(const float *albedo, const float *normal, const float *depth, const float *mv,
             const float *prev, int W, int H, float *in12, cudaStream_t stream) {
    const int64_t n = static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 4 * sm_count()));
    assemble_kernel<<<grid, 256, 0, stream>>>(albedo, normal, depth, mv, prev, n, in12);
    count_launch();
    return launch_status();
}

}  // namespace unet
}  // namespace spp

// ------------------------------------------------------------------ C ABI
using spp::aligned16;

namespace {
bool valid_net(int net) { return net >= 0 && net < spp::unet::kNumNets; }
bool aligned256(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }
}  // namespace

extern "C" int spp_net_spec(int net, int *cin, int *head0, int *head1, int *head2) {
    if (!valid_net(net) || !cin || !head0 || !head1 || !head2) return SPP_ERR_ARG;
    const spp::unet::NetSpec &n = spp::unet::kNets[net];
    *cin = n.cin;
    *head0 = n.heads[0];
    *head1 = n.heads[1];
    *head2 = n.heads[2];
    return SPP_OK;
}

extern "C" int spp_net_layer(int net, int i, int *cin, int *cout, int *relu) {
    if (!valid_net(net) || i < 0 || i >= spp::unet::kNumLayers || !cin || !cout || !relu)
        return SPP_ERR_ARG;
    const spp::unet::Layer l = spp::unet::layer(net, i);
    *cin = l.cin;
    *cout = l.cout;
    *relu = l.relu;
    return SPP_OK;
}

extern "C" int64_t spp_net_param_count(int net) {
    return valid_net(net) ? spp::unet::packed_layout(net, 0).param_count : -1;
}

extern "C" size_t spp_net_packed_bytes(int net, int with_backward) {
    return valid_net(net) ? spp::unet::packed_layout(net, with_backward).total : 0;
}

extern "C" int spp_net_pack(int net, const float *theta, int with_backward, void *packed,
                            size_t packed_bytes, cudaStream_t stream) {
    if (!valid_net(net) || !theta || !packed) return SPP_ERR_ARG;
    if (!aligned16(theta) || !aligned256(packed)) return SPP_ERR_ALIGN;
    if (packed_bytes < spp::unet::packed_layout(net, with_backward).total) return SPP_ERR_WORKSPACE;
    return spp::unet::pack(net, theta, with_backward, static_cast<unsigned char *>(packed), stream);
}

extern "C" size_t spp_net_workspace_bytes(int net, int B, int W, int H) {
    if (!valid_net(net) || B < 0 || W < 0 || H < 0) return 0;
    return spp::unet::act_layout(net, B, W, H).total;
}

extern "C" int spp_net_forward(int net, const void *packed, const float *in, int B, int W, int H,
                               float *head0, float *head1, float *head2, void *ws,
                               size_t ws_bytes, int32_t *status, cudaStream_t stream) {
    if (!valid_net(net) || B < 0 || W < 0 || H < 0 || !packed || !in || !head0 || !ws)
        return SPP_ERR_ARG;
    const spp::unet::NetSpec &n = spp::unet::kNets[net];
    if ((n.heads[1] && !head1) || (n.heads[2] && !head2)) return SPP_ERR_ARG;
    if (W % 4 || H % 4) return SPP_ERR_SHAPE;
    if (!aligned256(packed) || !aligned256(ws) || !aligned16(in) || !aligned16(head0) ||
        (n.heads[1] && !aligned16(head1)) || (n.heads[2] && !aligned16(head2)))
        return SPP_ERR_ALIGN;
    if (ws_bytes < spp::unet::act_layout(net, B, W, H).total) return SPP_ERR_WORKSPACE;
    if (static_cast<int64_t>(B) * W * H == 0) return SPP_OK;
    return spp::unet::forward(net, static_cast<const unsigned char *>(packed), in, B, W, H, nullptr,
                              head0, head1, head2, static_cast<unsigned char *>(ws), status,
                              stream);
}

extern "C" int spp_net_input_layout(int net, int B, int W, int H, size_t *offset,
                                    int *channels) {
    if (!valid_net(net) || B < 0 || W < 0 || H < 0 || !offset || !channels) return SPP_ERR_ARG;
    const spp::unet::ActLayout A = spp::unet::act_layout(net, B, W, H);
    *offset = A.xin;
    *channels = A.xin_c;
    return SPP_OK;
}

extern "C" int spp_net_forward_prepared(int net, const void *packed, int B, int W, int H,
                                        float *head0, float *head1, float *head2, void *ws,
                                        size_t ws_bytes, int32_t *status, cudaStream_t stream) {
    if (!valid_net(net) || B < 0 || W < 0 || H < 0 || !packed || !head0 || !ws)
        return SPP_ERR_ARG;
    const spp::unet::NetSpec &n = spp::unet::kNets[net];
    if ((n.heads[1] && !head1) || (n.heads[2] && !head2)) return SPP_ERR_ARG;
    if (W % 4 || H % 4) return SPP_ERR_SHAPE;
    if (!aligned256(packed) || !aligned256(ws) || !aligned16(head0) ||
        (n.heads[1] && !aligned16(head1)) || (n.heads[2] && !aligned16(head2)))
        return SPP_ERR_ALIGN;
    if (ws_bytes < spp::unet::act_layout(net, B, W, H).total) return SPP_ERR_WORKSPACE;
    if (static_cast<int64_t>(B) * W * H == 0) return SPP_OK;
    return spp::unet::forward(net, static_cast<const unsigned char *>(packed), nullptr, B, W, H,
                              nullptr, head0, head1, head2, static_cast<unsigned char *>(ws),
                              status, stream);
}

extern "C" size_t spp_density_softmax_workspace_bytes(int B) {
    return B < 0 ? 0 : static_cast<size_t>(std::max(B, 1)) * sizeof(uint32_t);
}

extern "C" int spp_density_softmax(const float *z, int B, int W, int H, int64_t batch_stride,
                                   float *density, void *ws, size_t ws_bytes,
                                   cudaStream_t stream) {
    if (!z || !density || !ws || B < 0 || W < 0 || H < 0 ||
        batch_stride < static_cast<int64_t>(W) * H)
        return SPP_ERR_ARG;
    if (!aligned16(z) || !aligned16(density) || !aligned16(ws)) return SPP_ERR_ALIGN;
    if (ws_bytes < static_cast<size_t>(std::max(B, 1)) * sizeof(uint32_t)) return SPP_ERR_WORKSPACE;
    if (static_cast<int64_t>(B) * W * H == 0) return SPP_OK;
    return spp::unet::density_softmax(z, B, static_cast<int64_t>(W) * H, batch_stride, density,
                                      static_cast<uint32_t *>(ws), stream);
}

// The joint predictor (network 0) under its original names.
extern "C" int spp_unet_layer(int i, int *cin, int *cout, int *relu) {
    return spp_net_layer(spp::unet::kNetJoint, i, cin, cout, relu);
}

extern "C" int64_t spp_unet_param_count(void) { return spp_net_param_count(spp::unet::kNetJoint); }

extern "C" size_t spp_unet_packed_bytes(int with_backward) {
    return spp_net_packed_bytes(spp::unet::kNetJoint, with_backward);
}

extern "C" int spp_unet_pack(const float *theta, int with_backward, void *packed,
                             size_t packed_bytes, cudaStream_t stream) {
    return spp_net_pack(spp::unet::kNetJoint, theta, with_backward, packed, packed_bytes, stream);
}

extern "C" int spp_assemble_features(const float *albedo, const float *normal, const float *depth,
                                     const float *mv, const float *prev_ldr, int W, int H,
                                     float *in12, cudaStream_t stream) {
    if (W < 0 || H < 0 || !albedo || !normal || !depth || !mv || !in12) return SPP_ERR_ARG;
    if (!aligned16(albedo) || !aligned16(normal) || !aligned16(depth) || !aligned16(mv) ||
        !aligned16(in12) || (prev_ldr && !aligned16(prev_ldr)))
        return SPP_ERR_ALIGN;
    return spp::unet::assemble(albedo, normal, depth, mv, prev_ldr, W, H, in12, stream);
}

extern "C" size_t spp_predict_workspace_bytes(int B, int W, int H) {
    return spp_net_workspace_bytes(spp::unet::kNetJoint, B, W, H);
}

extern "C" int spp_predict_density_and_kernels(const void *packed, const float *in12, int B, int W,
                                               int H, float *density, float *logits0,
                                               float *logits1, float *logits2, void *ws,
                                               size_t ws_bytes, int32_t *status,
                                               cudaStream_t stream) {
    if (B < 0 || W < 0 || H < 0 || !packed || !in12 || !density || !logits0 || !logits1 ||
        !logits2 || !ws)
        return SPP_ERR_ARG;
    if (W % 4 || H % 4) return SPP_ERR_SHAPE;
    if (!aligned256(packed) || !aligned256(ws) || !aligned16(in12) || !aligned16(density) ||
        !aligned16(logits0) || !aligned16(logits1) || !aligned16(logits2))
        return SPP_ERR_ALIGN;
    if (ws_bytes < spp::unet::act_layout(spp::unet::kNetJoint, B, W, H).total)
        return SPP_ERR_WORKSPACE;
    if (static_cast<int64_t>(B) * W * H == 0) return SPP_OK;
    return spp::unet::forward(spp::unet::kNetJoint, static_cast<const unsigned char *>(packed),
                              in12, B, W, H, density, logits0, logits1, logits2,
                              static_cast<unsigned char *>(ws), status, stream);
}

// ----------------------------------------------------- single conv layers
extern "C" size_t spp_conv3x3_workspace_bytes(int cin, int cout) {
    if (cin <= 0 || cout <= 0) return 0;
    using spp::unet::round16;
    return std::max(spp::conv::packed_bytes(round16(cin), round16(cout)),
                    spp::conv::packed_bytes(round16(cout), round16(cin)));
}

static int conv_layer_common(const void *in, int B, int W, int H, int cin_conv, int n_conv,
                             const float *w, void *out, void *ws, size_t ws_bytes) {
    if (B < 0 || W < 0 || H < 0 || cin_conv <= 0 || !in || !w || !out || !ws) return SPP_ERR_ARG;
    if (cin_conv % 8 || !spp::conv::supported_n(n_conv)) return SPP_ERR_ARG;
    if (!aligned16(in) || !aligned16(out) || !aligned16(w) || !aligned16(ws)) return SPP_ERR_ALIGN;
    if (ws_bytes < spp::conv::packed_bytes(spp::unet::round16(cin_conv), n_conv))
        return SPP_ERR_WORKSPACE;
    return SPP_OK;
}

extern "C" int spp_conv3x3_forward(const uint16_t *x, int B, int W, int H, int cin, int cout,
                                   const float *w, const float *bias, int relu, uint16_t *y,
                                   void *ws, size_t ws_bytes, int32_t *status,
                                   cudaStream_t stream) {
    int rc = conv_layer_common(x, B, W, H, cin, cout, w, y, ws, ws_bytes);
    if (rc != SPP_OK) return rc;
    const int cin_pad = spp::unet::round16(cin);
    auto *wp = static_cast<__nv_bfloat16 *>(ws);
    rc = spp::conv::pack_weights(w, cin, cout, 0, cin_pad, cout, wp, stream);
    if (rc != SPP_OK) return rc;
    spp::conv::ConvArgs a;
    a.B = B;
    a.H = H;
    a.W = W;
    a.cin_pad = cin_pad;
    a.n = cout;
    a.cout = cout;
    a.src_mode = spp::conv::kSrcNHWC;
    a.src0 = reinterpret_cast<const __nv_bfloat16 *>(x);
    a.c0 = cin;
    a.wpack = wp;
    a.bias = bias;
    a.epi_mode = relu ? spp::conv::kEpiReluBF16 : spp::conv::kEpiBF16;
    a.out = reinterpret_cast<__nv_bfloat16 *>(y);
    a.status = status;
    return spp::conv::conv3x3(a, stream);
}

extern "C" int spp_conv3x3_backward_data(const uint16_t *g, int B, int W, int H, int cin, int cout,
                                         const float *w, const uint16_t *act, uint16_t *gx,
                                         void *ws, size_t ws_bytes, int32_t *status,
                                         cudaStream_t stream) {
    int rc = conv_layer_common(g, B, W, H, cout, cin, w, gx, ws, ws_bytes);
    if (rc != SPP_OK) return rc;
    if (act && !aligned16(act)) return SPP_ERR_ALIGN;
    const int cin_pad = spp::unet::round16(cout);
    auto *wp = static_cast<__nv_bfloat16 *>(ws);
    rc = spp::conv::pack_weights(w, cin, cout, 1, cin_pad, cin, wp, stream);
    if (rc != SPP_OK) return rc;
    spp::conv::ConvArgs a;
    a.B = B;
    a.H = H;
    a.W = W;
    a.cin_pad = cin_pad;
    a.n = cin;
    a.cout = cin;
    a.src_mode = spp::conv::kSrcNHWC;
    a.src0 = reinterpret_cast<const __nv_bfloat16 *>(g);
    a.c0 = cout;
    a.wpack = wp;
    a.epi_mode = act ? spp::conv::kEpiMaskBF16 : spp::conv::kEpiBF16;
    a.act = reinterpret_cast<const __nv_bfloat16 *>(act);
    a.out = reinterpret_cast<__nv_bfloat16 *>(gx);
    a.status = status;
    return spp::conv::conv3x3(a, stream);
}
