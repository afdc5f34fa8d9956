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

struct Layer {
    int cin, cout, relu;
};
extern const Layer kLayers[kNumLayers];

// Layer indices.
enum : int { E0A, E0B, E1A, E1B, E2A, E2B, H2, D1A, D1B, H1, D0A, D0B, H0 };

int round16(int c);
int fwd_n(int i);

// Byte offsets inside the packed parameter blob and element offsets in theta.
struct PackedLayout {
    size_t fwd[kNumLayers];   // BF16 forward operand
    size_t bias[kNumLayers];  // FP32 bias, padded to fwd_n
    size_t bwd[kNumLayers];   // BF16 data-gradient operand (0 if absent)
    int64_t theta_w[kNumLayers], theta_b[kNumLayers];
    int64_t param_count;
    size_t total;
};
PackedLayout packed_layout(int with_backward);

// Byte offsets of the BF16 NHWC activations inside the forward workspace.
struct ActLayout {
    size_t x16;  // the input features, BF16 [B][H][W][16] (channels 12..15 zero)
    size_t e0a, s0, p0, e1a, s1, p1, e2a, bt, d1a, t1, d0a, t0;  // p0, p1: 2x2 pools of s0, s1
    size_t zmax;
    size_t total;
};
ActLayout act_layout(int B, int W, int H);

// Input of layer i as its convolution reads it (grid, source mode, pointers
// into the forward workspace `ws`, cin_pad); the caller fills the rest.
conv::ConvArgs layer_input(int i, int B, int W, int H, const float *in12,
                           const unsigned char *ws);
// Byte offset of layer i's BF16 output in the forward workspace (heads: -1).
size_t layer_output(int i, const ActLayout &A);

int forward(const unsigned char *packed, const float *in12, int B, int W, int H, float *density,
            float *logits0, float *logits1, float *logits2, unsigned char *ws, int32_t *status,
            cudaStream_t stream);
size_t backward_workspace_bytes(int B, int W, int H);
int backward(const unsigned char *packed, const float *in12, int B, int W, int H,
             const unsigned char *fws, const float *g0, const float *g1, const float *g2,
             float *grad_theta, unsigned char *bws, int32_t *status, cudaStream_t stream);
int adamw(float *theta, const float *grad, float *m, float *v, int64_t n, int step, float lr,
          float b1, float b2, float eps, float wd, float grad_scale, cudaStream_t stream);
int pack(const float *theta, int with_backward, unsigned char *packed, cudaStream_t stream);
int assemble(const float *albedo, const float *normal, const float *depth, const float *mv,
             const float *prev, int W, int H, float *in12, cudaStream_t stream);

}  // namespace unet
}  // namespace spp
