// Host-side interface of the tensor-core 3x3 convolution kernels
// (conv_tc.cu) used by the predictor network (unet.cu) and the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace spp {
namespace conv {

// Where the K operand (the input channels of the convolution) comes from.
enum SrcMode : int {
    kSrcNHWC = 0,       // src0: BF16 [B][H][W][c0]
    kSrcPool = 1,       // src0: BF16 [B][2H][2W][c0], 2x2 average taken on load
    kSrcConcatUp = 2,   // channels [0,c0) from src0 [B][H][W][c0], then [c0,c0+c1)
                        // from src1 [B][H/2][W/2][c1] upsampled (nearest)
    kSrcPlanarF32 = 3,  // srcf: FP32 [B][cf][H][W]
};

// What the epilogue does with the FP32 accumulator of output channel n.
enum EpiMode : int {
    kEpiReluBF16 = 0,   // out[b][y][x][n] = bf16(max(acc + bias[n], 0))
    kEpiF32Planar = 1,  // outf[b][n][y][x] = acc + bias[n], n < cout
    kEpiMaskBF16 = 2,   // out[b][y][x][n] = bf16(acc * (act[b][y][x][n] > 0))
    kEpiBF16 = 3,       // out[b][y][x][n] = bf16(acc + bias[n]), bias optional
};

struct ConvArgs {
    int B = 0, H = 0, W = 0;  // output grid (the input grid of the convolution)
    int cin_pad = 0;          // input channels padded to a multiple of 16
    int n = 0;                // output channels padded (16..192, the MMA N)
    int cout = 0;             // real output channels (F32 planar epilogue)
    int src_mode = kSrcNHWC;
    const __nv_bfloat16 *src0 = nullptr;
    int c0 = 0;
    const __nv_bfloat16 *src1 = nullptr;
    int c1 = 0;
    const float *srcf = nullptr;
    int cf = 0;
    const __nv_bfloat16 *wpack = nullptr;  // pack_weights() layout for (cin_pad, n)
    const float *bias = nullptr;           // [cout] or null (zero)
    int epi_mode = kEpiReluBF16;
    __nv_bfloat16 *out = nullptr;          // NHWC, channel stride n
    const __nv_bfloat16 *act = nullptr;    // kEpiMaskBF16: NHWC, channel stride n
    float *outf = nullptr;                 // [B][cout][H][W]
    // kEpiReluBF16 only: also write the 2x2 average of the stored BF16 values
    // to pool_out [B][H/2][W/2][n] (H and W even)
    __nv_bfloat16 *pool_out = nullptr;
    int tma_out = 0;  // set by the launcher: FP32 planar output through TMA stores
    int tma_in = 0;   // set by the launcher: NHWC halo through TMA loads (1), or only the
                      // skip-connection chunks of an upsampling layer (2), or those and
                      // the coarse rows of its upsampled chunks, expanded in shared
                      // memory (3)
    int32_t *status = nullptr;
};

// Bytes of a packed weight operand for a convolution with cin_pad input and n
// output channels: BF16 [cin_pad/16][9 taps][2][n][8]; for n = 32 the taps of
// one dx are stacked along N instead: [cin_pad/16][3 dx][2][96 = dy 2,1,0 x 32][8]
// (the same size).
inline size_t packed_bytes(int cin_pad, int n) {
    return static_cast<size_t>(cin_pad / 16) * 9 * 2 * n * 8 * 2;
}

// Packs FP32 weights w [cout][cin][3][3] for the forward convolution
// (transpose = 0: input channel = cin, output = cout) or for its data
// gradient (transpose = 1: the kernel flipped, input channel = cout,
// output = cin).  Padding entries are zero.
int pack_weights(const float *w, int cin, int cout, int transpose, int cin_pad, int n,
                 __nv_bfloat16 *dst, cudaStream_t stream);

// Runs the convolution; returns SPP_OK or an SPP error code.
int conv3x3(const ConvArgs &a, cudaStream_t stream);

// Weight gradient (wgrad_tc.cu).  x describes the layer's input exactly as
// the forward convolution reads it (B, H, W, cin_pad and the source mode);
// g the gradient with respect to the layer's output before its ReLU
// (kSrcNHWC with c0 = its channel count, or kSrcPlanarF32 with cf = cout),
// on the same grid.  gw [cout][cin][3][3] and gb [cout] are overwritten.
struct WgradArgs {
    ConvArgs x;
    ConvArgs g;
    int cin = 0, cout = 0;  // real channel counts
    int n = 0;              // cout padded: 32, 64 or 128 (the MMA N)
    float *partial = nullptr;
    float *pbias = nullptr;
    int32_t *status = nullptr;
};
int wgrad_splits(int B, int W, int H, int cin_pad);
size_t wgrad_workspace_bytes(int B, int W, int H, int cin_pad, int n);
int wgrad(const WgradArgs &a, float *gw, float *gb, void *ws, cudaStream_t stream);

// Supported MMA widths of conv3x3.
inline bool supported_n(int n) {
    return n == 16 || n == 32 || n == 64 || n == 96 || n == 128 || n == 192;
}

}  // namespace conv
}  // namespace spp
