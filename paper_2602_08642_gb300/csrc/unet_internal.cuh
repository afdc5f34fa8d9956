// Layer table and memory layouts of the predictor network (unet.cu and
// its backward, unet_train.cu).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

#include "conv_tc.cuh"

namespace spp {
namespace unet {

constexpr int kNumLayers = 13;
constexpr int kDensityChannel = 54;

// Network specifications (the layer table of each is fixed by its input
// channels and head widths):
//   kNetJoint     12 inputs, h0 = 54 kernel logits + density logit, h1 29, h2 25
//   kNetSampler   19 inputs (12 + 7 latents), h0 = density logit, no h1 / h2
//   kNetDenoiser  24 inputs, h0 = 54 logits + 3 demodulation + 7 latents, h1 29, h2 25
enum : int { kNetJoint = 0, kNetSampler = 1, kNetDenoiser = 2, kNumNets = 3 };
struct NetSpec {
    int cin;
    int heads[3];  // output channels of h0, h1, h2 (0 = absent)
};
extern const NetSpec kNets[kNumNets];

struct Layer {
    int cin, cout, relu;  // cout = 0: the head is absent in this network
};

// Layer indices (slots; a network without h1 / h2 leaves them empty).
enum : int { E0A, E0B, E1A, E1B, E2A, E2B, H2, D1A, D1B, H1, D0A, D0B, H0 };

Layer layer(int net, int i);
inline bool present(int net, int i) { return layer(net, i).cout > 0; }
int level_of(int i);
int round16(int c);
int fwd_n(int net, int i);
int input_channels_padded(int net);  // channels of the BF16 NHWC input copy

// Byte offsets inside the packed parameter blob and element offsets in theta.
struct PackedLayout {
    size_t fwd[kNumLayers];   // BF16 forward operand
    size_t bias[kNumLayers];  // FP32 bias, padded to fwd_n
    size_t bwd[kNumLayers];   // BF16 data-gradient operand (0 if absent)
    int64_t theta_w[kNumLayers], theta_b[kNumLayers];
    int64_t param_count;
    size_t total;
};
PackedLayout packed_layout(int net, int with_backward);

// Byte offsets of the BF16 NHWC activations inside the forward workspace.
struct ActLayout {
    size_t xin;  // the input features, BF16 [B][H][W][xin_c] (padding channels zero)
    int xin_c;
    size_t e0a, s0, p0, e1a, s1, p1, e2a, bt, d1a, t1, d0a, t0;  // p0, p1: 2x2 pools of s0, s1
    size_t zmax;
    size_t total;
};
ActLayout act_layout(int net, int B, int W, int H);

// Input of layer i as its convolution reads it (grid, source mode, pointers
// into the forward workspace `ws`, cin_pad); the caller fills the rest.
conv::ConvArgs layer_input(int net, int i, int B, int W, int H, const unsigned char *ws);
// Byte offset of layer i's BF16 output in the forward workspace (heads: -1).
size_t layer_output(int i, const ActLayout &A);

// Forward of network `net` on in [B][cin][H][W] FP32: heads written as FP32
// planar [B][c][H>>l][W>>l] (absent heads: pointer unused).  The joint
// network also writes the unnormalised density exp(z - max z) if density
// is not null.
int forward(int net, const unsigned char *packed, const float *in, int B, int W, int H,
            float *density, float *head0, float *head1, float *head2, unsigned char *ws,
            int32_t *status, cudaStream_t stream);
size_t backward_workspace_bytes(int net, int B, int W, int H);
// Parameter gradients (overwritten) and, if grad_in is not null, the
// gradient with respect to the FP32 input [B][cin][H][W].
int backward(int net, const unsigned char *packed, int B, int W, int H, const unsigned char *fws,
             const float *g0, const float *g1, const float *g2, float *grad_theta, float *grad_in,
             unsigned char *bws, int32_t *status, cudaStream_t stream);
int adamw(float *theta, const float *grad, float *m, float *v, int64_t n, int step, float lr,
          float b1, float b2, float eps, float wd, float grad_scale, cudaStream_t stream);
int pack(int net, const float *theta, int with_backward, unsigned char *packed,
         cudaStream_t stream);
int assemble(const float *albedo, const float *normal, const float *depth, const float *mv,
             const float *prev, int W, int H, float *in12, cudaStream_t stream);
int density_softmax(const float *z, int B, int64_t hw, int64_t batch_stride, float *d,
                    uint32_t *zmax, cudaStream_t stream);

}  // namespace unet
}  // namespace spp
