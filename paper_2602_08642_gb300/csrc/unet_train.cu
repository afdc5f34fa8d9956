// Backward of the predictor network and its optimiser (training, Sec. 6.3):
// data gradients on the tensor cores through conv_tc.cu (flipped,
// transposed weights; the ReLU mask of the layer below fused into the
// epilogue), weight gradients through wgrad_tc.cu, the gradient junctions
// of the pooling / upsampling / concatenation edges in one small kernel,
// and AdamW on the FP32 master parameters.
#include <cuda_bf16.h>

#include <algorithm>

#include "conv_src.cuh"
#include "conv_tc.cuh"
#include "spp_internal.cuh"
#include "unet_internal.cuh"

namespace spp {
namespace unet {
namespace {

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// BF16 NHWC gradient buffers of the backward.
struct GradLayout {
    size_t d0b, d0a, cat0, e0b, e0a, gin;          // level 0 (gin: input gradient)
    size_t t1h, d1b, d1a, cat1, e1b, e1a, pool0;   // level 1
    size_t bth, e2b, e2a, pool1;                   // level 2
    size_t wg;                                     // weight-gradient scratch
    size_t total;
};

GradLayout grad_layout(int net, int B, int W, int H) {
    GradLayout G{};
    const size_t p0 = static_cast<size_t>(B) * H * W, p1 = p0 / 4, p2 = p0 / 16;
    size_t off = 0;
    auto take = [&](size_t elems) {
        const size_t o = off;
        off = align256(off + elems * sizeof(__nv_bfloat16));
        return o;
    };
    G.d0b = take(p0 * 32);
    G.d0a = take(p0 * 32);
    G.cat0 = take(p0 * 96);
    G.e0b = take(p0 * 32);
    G.e0a = take(p0 * 32);
    G.gin = take(p0 * input_channels_padded(net));
    G.t1h = take(p1 * 64);
    G.d1b = take(p1 * 64);
    G.d1a = take(p1 * 64);
    G.cat1 = take(p1 * 192);
    G.e1b = take(p1 * 64);
    G.e1a = take(p1 * 64);
    G.pool0 = take(p1 * 32);
    G.bth = take(p2 * 128);
    G.e2b = take(p2 * 128);
    G.e2a = take(p2 * 128);
    G.pool1 = take(p2 * 64);
    G.wg = off;
    size_t wg = 0;
    for (int i = 0; i < kNumLayers; ++i) {
        if (!present(net, i)) continue;
        const int level = level_of(i);
        const int cin_pad = i == E0A ? input_channels_padded(net) : round16(layer(net, i).cin);
        wg = std::max(wg, conv::wgrad_workspace_bytes(B, W >> level, H >> level, cin_pad,
                                                      fwd_n(net, i)));
    }
    G.total = align256(off + wg);
    return G;
}

// out[p][c] = (act[p][c] > 0) * (A[p][a_off + c] + sum over the 2x2 fine
// pixels of F[.][f_off + c] + Cq[p/2][c] / 4), each term optional; 8
// channels per thread.
__global__ void junction_kernel(int B, int H, int W, int C, const __nv_bfloat16 *__restrict__ act,
                                const __nv_bfloat16 *__restrict__ A, int a_c, int a_off,
                                const __nv_bfloat16 *__restrict__ F, int f_c, int f_off,
                                const __nv_bfloat16 *__restrict__ Cq, int c_c,
                                __nv_bfloat16 *__restrict__ out) {
    using conv::ldg16;
    using conv::pack_bf16x2;
    using conv::unpack_bf16x2;
    const int c8 = C / 8;
    const int64_t total = static_cast<int64_t>(B) * H * W * c8;
    for (int64_t idx = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int c = static_cast<int>(idx % c8) * 8;
        const int64_t p = idx / c8;
        const int x = static_cast<int>(p % W);
        const int y = static_cast<int>((p / W) % H);
        const int b = static_cast<int>(p / (static_cast<int64_t>(W) * H));
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0.f;
        auto add = [&](uint4 q, float s) {
            const uint32_t *u = &q.x;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = unpack_bf16x2(u[k]);
                v[2 * k] += s * f.x;
                v[2 * k + 1] += s * f.y;
            }
        };
        if (A) add(ldg16(A + p * a_c + a_off + c), 1.f);
        if (F) {
            const int Wf = 2 * W;
            const int64_t f0 = (static_cast<int64_t>(b) * 2 * H + 2 * y) * Wf + 2 * x;
            add(ldg16(F + f0 * f_c + f_off + c), 1.f);
            add(ldg16(F + (f0 + 1) * f_c + f_off + c), 1.f);
            add(ldg16(F + (f0 + Wf) * f_c + f_off + c), 1.f);
            add(ldg16(F + (f0 + Wf + 1) * f_c + f_off + c), 1.f);
        }
        if (Cq) {
            const int64_t q = (static_cast<int64_t>(b) * (H / 2) + y / 2) * (W / 2) + x / 2;
            add(ldg16(Cq + q * c_c + c), 0.25f);
        }
        const uint4 m = ldg16(act + p * C + c);
        const uint32_t *mu = &m.x;
        uint32_t o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 mv = unpack_bf16x2(mu[k]);
            o[k] = pack_bf16x2(mv.x > 0.f ? v[2 * k] : 0.f, mv.y > 0.f ? v[2 * k + 1] : 0.f);
        }
        *reinterpret_cast<uint4 *>(out + p * C + c) = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

__global__ void adamw_kernel(float *__restrict__ theta, const float *__restrict__ grad,
                             float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                             float b1, float b2, float eps, float wd, float grad_scale, float c1,
                             float c2) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float g = grad[i] * grad_scale;
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / c1, vh = vi / c2;
        theta[i] -= lr * (mh / (sqrtf(vh) + eps) + wd * theta[i]);
    }
}

// BF16 NHWC [B][H][W][CP] -> FP32 planar [B][C][H][W] (the first C channels).
__global__ void nhwc_to_planar_kernel(const __nv_bfloat16 *__restrict__ src, int CP, int C,
                                      int64_t n, int64_t hw, float *__restrict__ dst) {
    for (int64_t p = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; p < n;
         p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t b = p / hw, i = p - b * hw;
        const __nv_bfloat16 *s = src + p * CP;
        float *d = dst + b * C * hw + i;
        for (int c = 0; c < C; ++c) d[c * hw] = __bfloat162float(s[c]);
    }
}

int launch_junction(int B, int H, int W, int C, const __nv_bfloat16 *act, const __nv_bfloat16 *A,
                    int a_c, int a_off, const __nv_bfloat16 *F, int f_c, int f_off,
                    const __nv_bfloat16 *Cq, int c_c, __nv_bfloat16 *out, cudaStream_t stream) {
    const int64_t total = static_cast<int64_t>(B) * H * W * (C / 8);
    if (total == 0) return SPP_OK;
    const int grid = static_cast<int>(std::min<int64_t>((total + 255) / 256, 8 * sm_count()));
    junction_kernel<<<grid, 256, 0, stream>>>(B, H, W, C, act, A, a_c, a_off, F, f_c, f_off, Cq,
                                              c_c, out);
    count_launch();
    return launch_status();
}

}  // namespace

size_t backward_workspace_bytes(int net, int B, int W, int H) {
    return grad_layout(net, B, W, H).total;
}

int backward(int net, const unsigned char *packed, int B, int W, int H, const unsigned char *fws,
             const float *g0, const float *g1, const float *g2, float *grad_theta, float *grad_in,
             unsigned char *bws, int32_t *status, cudaStream_t stream) {
    const PackedLayout P = packed_layout(net, 1);
    const ActLayout A = act_layout(net, B, W, H);
    const GradLayout G = grad_layout(net, B, W, H);
    auto act = [&](size_t off) { return reinterpret_cast<const __nv_bfloat16 *>(fws + off); };
    auto gb = [&](size_t off) { return reinterpret_cast<__nv_bfloat16 *>(bws + off); };
    const float *gheads[kNumLayers] = {};
    gheads[H0] = g0;
    gheads[H1] = g1;
    gheads[H2] = g2;
    const bool has_h1 = present(net, H1), has_h2 = present(net, H2);
    // gradient with respect to each layer's pre-activation output
    size_t gpre[kNumLayers] = {G.e0a, G.e0b, G.e1a, G.e1b, G.e2a, G.e2b, 0,
                               G.d1a, G.d1b, 0,     G.d0a, G.d0b, 0};
    int rc = SPP_OK;

    auto gsrc = [&](int i, int level) {
        conv::ConvArgs g;
        g.B = B;
        g.W = W >> level;
        g.H = H >> level;
        const Layer l = layer(net, i);
        if (!l.relu) {
            g.src_mode = conv::kSrcPlanarF32;
            g.srcf = gheads[i];
            g.cf = l.cout;
        } else {
            g.src_mode = conv::kSrcNHWC;
            g.src0 = gb(gpre[i]);
            g.c0 = l.cout;
        }
        return g;
    };
    auto wgrad_layer = [&](int i) {
        if (rc != SPP_OK || !present(net, i)) return;
        const Layer l = layer(net, i);
        conv::WgradArgs w;
        w.x = layer_input(net, i, B, W, H, fws);
        w.g = gsrc(i, level_of(i));
        w.cin = l.cin;
        w.cout = l.cout;
        w.n = fwd_n(net, i);
        w.status = status;
        rc = conv::wgrad(w, grad_theta + P.theta_w[i], grad_theta + P.theta_b[i], bws + G.wg,
                         stream);
    };
    // data gradient of layer i into `out` (channels cin, the input layer's
    // padded), masked by `mask`
    auto dgrad_layer = [&](int i, __nv_bfloat16 *out, const __nv_bfloat16 *mask) {
        if (rc != SPP_OK || !present(net, i)) return;
        const Layer l = layer(net, i);
        const int level = level_of(i);
        conv::ConvArgs a = gsrc(i, level);
        a.cin_pad = round16(l.cout);
        a.n = i == E0A ? input_channels_padded(net) : l.cin;
        a.cout = a.n;
        a.wpack = reinterpret_cast<const __nv_bfloat16 *>(packed + P.bwd[i]);
        a.epi_mode = mask ? conv::kEpiMaskBF16 : conv::kEpiBF16;
        a.act = mask;
        a.out = out;
        a.status = status;
        rc = conv::conv3x3(a, stream);
    };
    auto junction = [&](int level, int C, const __nv_bfloat16 *actv, const __nv_bfloat16 *Ain,
                        int a_c, int a_off, const __nv_bfloat16 *F, int f_c, int f_off,
                        const __nv_bfloat16 *Cq, int c_c, __nv_bfloat16 *out) {
        if (rc != SPP_OK) return;
        rc = launch_junction(B, H >> level, W >> level, C, actv, Ain, a_c, a_off, F, f_c, f_off, Cq,
                             c_c, out, stream);
    };

    // decoder, level 0
    wgrad_layer(H0);
    dgrad_layer(H0, gb(G.d0b), act(A.t0));
    wgrad_layer(D0B);
    dgrad_layer(D0B, gb(G.d0a), act(A.d0a));
    wgrad_layer(D0A);
    dgrad_layer(D0A, gb(G.cat0), nullptr);
    // decoder, level 1
    wgrad_layer(H1);
    dgrad_layer(H1, gb(G.t1h), nullptr);
    junction(1, 64, act(A.t1), has_h1 ? gb(G.t1h) : nullptr, 64, 0, gb(G.cat0), 96, 32, nullptr,
             0, gb(G.d1b));
    wgrad_layer(D1B);
    dgrad_layer(D1B, gb(G.d1a), act(A.d1a));
    wgrad_layer(D1A);
    dgrad_layer(D1A, gb(G.cat1), nullptr);
    // bottleneck, level 2
    wgrad_layer(H2);
    dgrad_layer(H2, gb(G.bth), nullptr);
    junction(2, 128, act(A.bt), has_h2 ? gb(G.bth) : nullptr, 128, 0, gb(G.cat1), 192, 64,
             nullptr, 0, gb(G.e2b));
    wgrad_layer(E2B);
    dgrad_layer(E2B, gb(G.e2a), act(A.e2a));
    wgrad_layer(E2A);
    dgrad_layer(E2A, gb(G.pool1), nullptr);
    // encoder, level 1
    junction(1, 64, act(A.s1), gb(G.cat1), 192, 0, nullptr, 0, 0, gb(G.pool1), 64, gb(G.e1b));
    wgrad_layer(E1B);
    dgrad_layer(E1B, gb(G.e1a), act(A.e1a));
    wgrad_layer(E1A);
    dgrad_layer(E1A, gb(G.pool0), nullptr);
    // encoder, level 0
    junction(0, 32, act(A.s0), gb(G.cat0), 96, 0, nullptr, 0, 0, gb(G.pool0), 32, gb(G.e0b));
    wgrad_layer(E0B);
    dgrad_layer(E0B, gb(G.e0a), act(A.e0a));
    wgrad_layer(E0A);
    if (grad_in && rc == SPP_OK) {
        dgrad_layer(E0A, gb(G.gin), nullptr);
        if (rc != SPP_OK) return rc;
        const int64_t n = static_cast<int64_t>(B) * W * H;
        const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 8 * sm_count()));
        nhwc_to_planar_kernel<<<grid, 256, 0, stream>>>(gb(G.gin), A.xin_c, kNets[net].cin, n,
                                                        static_cast<int64_t>(W) * H, grad_in);
        count_launch();
        rc = launch_status();
    }
    return rc;
}

int adamw(float *theta, const float *grad, float *m, float *v, int64_t n, int step, float lr,
          float b1, float b2, float eps, float wd, float grad_scale, cudaStream_t stream) {
    if (n == 0) return SPP_OK;
    const float c1 = 1.f - powf(b1, static_cast<float>(step));
    const float c2 = 1.f - powf(b2, static_cast<float>(step));
    const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 4 * sm_count()));
    adamw_kernel<<<grid, 256, 0, stream>>>(theta, grad, m, v, n, lr, b1, b2, eps, wd, grad_scale,
                                           c1, c2);
    count_launch();
    return launch_status();
}

}  // namespace unet
}  // namespace spp

// ------------------------------------------------------------------ C ABI
using spp::aligned16;

extern "C" size_t spp_net_backward_workspace_bytes(int net, int B, int W, int H) {
    if (net < 0 || net >= spp::unet::kNumNets || B < 0 || W < 0 || H < 0) return 0;
    return spp::unet::backward_workspace_bytes(net, B, W, H);
}

extern "C" int spp_net_backward(int net, const void *packed, int B, int W, int H,
                                const void *fwd_ws, size_t fwd_ws_bytes, const float *grad_head0,
                                const float *grad_head1, const float *grad_head2,
                                float *grad_theta, float *grad_in, void *ws, size_t ws_bytes,
                                int32_t *status, cudaStream_t stream) {
    if (net < 0 || net >= spp::unet::kNumNets || B < 0 || W < 0 || H < 0 || !packed || !fwd_ws ||
        !grad_head0 || !grad_theta || !ws)
        return SPP_ERR_ARG;
    const spp::unet::NetSpec &n = spp::unet::kNets[net];
    if ((n.heads[1] && !grad_head1) || (n.heads[2] && !grad_head2)) return SPP_ERR_ARG;
    if (W % 4 || H % 4) return SPP_ERR_SHAPE;
    auto a256 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; };
    if (!a256(packed) || !a256(fwd_ws) || !a256(ws) || !aligned16(grad_head0) ||
        (n.heads[1] && !aligned16(grad_head1)) || (n.heads[2] && !aligned16(grad_head2)) ||
        !aligned16(grad_theta) || (grad_in && !aligned16(grad_in)))
        return SPP_ERR_ALIGN;
    if (fwd_ws_bytes < spp::unet::act_layout(net, B, W, H).total ||
        ws_bytes < spp::unet::backward_workspace_bytes(net, B, W, H))
        return SPP_ERR_WORKSPACE;
    return spp::unet::backward(net, static_cast<const unsigned char *>(packed), B, W, H,
                               static_cast<const unsigned char *>(fwd_ws), grad_head0, grad_head1,
                               grad_head2, grad_theta, grad_in, static_cast<unsigned char *>(ws),
                               status, stream);
}

extern "C" size_t spp_unet_backward_workspace_bytes(int B, int W, int H) {
    return spp_net_backward_workspace_bytes(spp::unet::kNetJoint, B, W, H);
}

extern "C" int spp_unet_backward(const void *packed, const float *in12, int B, int W, int H,
                                 const void *fwd_ws, size_t fwd_ws_bytes, const float *grad_logits0,
                                 const float *grad_logits1, const float *grad_logits2,
                                 float *grad_theta, void *ws, size_t ws_bytes, int32_t *status,
                                 cudaStream_t stream) {
    if (!in12) return SPP_ERR_ARG;
    if (!aligned16(in12)) return SPP_ERR_ALIGN;
    return spp_net_backward(spp::unet::kNetJoint, packed, B, W, H, fwd_ws, fwd_ws_bytes,
                            grad_logits0, grad_logits1, grad_logits2, grad_theta, nullptr, ws,
                            ws_bytes, status, stream);
}

extern "C" int spp_adamw_step(float *theta, const float *grad, float *m, float *v, int64_t n,
                              int step, float lr, float beta1, float beta2, float eps,
                              float weight_decay, float grad_scale, cudaStream_t stream) {
    if (n < 0 || step < 1 || !theta || !grad || !m || !v) return SPP_ERR_ARG;
    if (!aligned16(theta) || !aligned16(grad) || !aligned16(m) || !aligned16(v)) return SPP_ERR_ALIGN;
    return spp::unet::adamw(theta, grad, m, v, n, step, lr, beta1, beta2, eps, weight_decay,
                            grad_scale, stream);
}

static int wgrad_n(int cout) { return cout <= 32 ? 32 : cout <= 64 ? 64 : 128; }

extern "C" size_t spp_conv3x3_backward_weights_workspace_bytes(int B, int W, int H, int cin,
                                                               int cout) {
    if (B < 0 || W < 0 || H < 0 || cin <= 0 || cout <= 0 || cout > 128) return 0;
    return spp::conv::wgrad_workspace_bytes(B, W, H, spp::unet::round16(cin), wgrad_n(cout));
}

extern "C" int spp_conv3x3_backward_weights(const uint16_t *x, const uint16_t *g, int B, int W,
                                            int H, int cin, int cout, float *gw, float *gb,
                                            void *ws, size_t ws_bytes, int32_t *status,
                                            cudaStream_t stream) {
    if (B < 0 || W < 0 || H < 0 || cin <= 0 || cout <= 0 || cout > 128 || !x || !g || !gw || !ws)
        return SPP_ERR_ARG;
    if (cin % 8 || cout % 8) return SPP_ERR_ARG;
    if (!aligned16(x) || !aligned16(g) || !aligned16(ws)) return SPP_ERR_ALIGN;
    if (ws_bytes < spp::conv::wgrad_workspace_bytes(B, W, H, spp::unet::round16(cin), wgrad_n(cout)))
        return SPP_ERR_WORKSPACE;
    spp::conv::WgradArgs a;
    a.x.B = a.g.B = B;
    a.x.W = a.g.W = W;
    a.x.H = a.g.H = H;
    a.x.cin_pad = spp::unet::round16(cin);
    a.x.src_mode = spp::conv::kSrcNHWC;
    a.x.src0 = reinterpret_cast<const __nv_bfloat16 *>(x);
    a.x.c0 = cin;
    a.g.src_mode = spp::conv::kSrcNHWC;
    a.g.src0 = reinterpret_cast<const __nv_bfloat16 *>(g);
    a.g.c0 = cout;
    a.cin = cin;
    a.cout = cout;
    a.n = wgrad_n(cout);
    a.status = status;
    return spp::conv::wgrad(a, gw, gb, ws, stream);
}
