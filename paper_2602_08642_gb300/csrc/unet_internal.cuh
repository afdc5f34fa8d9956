// Layer table and memory layouts of the predictor network (unet.cu and
// its backward, unet_train.cu).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime.h>

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
    size_t e0a, s0, e1a, s1, e2a, bt, d1a, t1, d0a, t0;
    size_t zmax;
    size_t total;
};
ActLayout act_layout(int B, int W, int H);

int forward(const unsigned char *packed, const float *in12, int B, int W, int H, float *density,
            float *logits0, float *logits1, float *logits2, unsigned char *ws, int32_t *status,
            cudaStream_t stream);
int pack(const float *theta, int with_backward, unsigned char *packed, cudaStream_t stream);
int assemble(const float *albedo, const float *normal, const float *depth, const float *mv,
             const float *prev, int W, int H, float *in12, cudaStream_t stream);

}  // namespace unet
}  // namespace spp
