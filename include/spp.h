/*
 * spp.h -- C ABI of the GB300 (sm_103a) library for sub-1-spp adaptive
 * sampling and gather-pyramid reconstruction, after "Forget Superresolution,
 * Sample Adaptively (when Path Tracing)" (arXiv 2602.08642).
 *
 * Conventions shared by every entry point
 *   - Images are planar FP32 [C][H][W], row-major, x fastest.  Level l of the
 *     pyramid is (W >> l) x (H >> l); W and H must be divisible by 2^(L-1).
 *   - Every data pointer is a DEVICE pointer owned by the caller, 16-byte
 *     aligned (SPP_ERR_ALIGN otherwise).  Arrays of pointers (layers, logits)
 *     are HOST arrays of device pointers.  The library allocates nothing:
 *     scratch space is a caller-provided workspace whose size the
 *     *_workspace_bytes queries return.
 *   - Every call is asynchronous on the given cudaStream_t and returns an int:
 *     SPP_OK, or a negative SPP_ERR_* for errors found on the host (no work is
 *     enqueued then).  Errors found by the kernels (bad density values, too
 *     small sample capacity, a look-back wait that gave up) are written to a
 *     caller-provided device int32 status word, first error wins; read it with
 *     spp_get_status and reset it with spp_clear_status.
 *   - Calls are thread-compatible: concurrent calls must use distinct
 *     workspaces and outputs.
 */
#ifndef SPP_H
#define SPP_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define SPP_OK 0
#define SPP_ERR_ARG (-1)       /* bad argument: null pointer, size out of range */
#define SPP_ERR_ALIGN (-2)     /* a pointer is not 16-byte aligned */
#define SPP_ERR_SHAPE (-3)     /* W or H not divisible by 2^(L-1), or L out of [2,5] */
#define SPP_ERR_WORKSPACE (-4) /* workspace too small */
#define SPP_ERR_CAPACITY (-5)  /* more samples than the sample buffers hold */
#define SPP_ERR_TIMEOUT (-6)   /* a bounded device-side wait gave up */
#define SPP_ERR_INPUT (-7)     /* density has NaN, inf, negative values, or sums to 0 */
#define SPP_ERR_CUDA (-8)      /* a CUDA runtime call failed */

/* Holdout weighting of the extra sample. */
#define SPP_HOLDOUT_RAMP 0 /* relaxed ramp of Eq. relaxed_holdout with h of Eq. h_factor */
#define SPP_HOLDOUT_HARD 1 /* hard step of Eq. holdout (the lambda -> inf limit), weight 1 */
/* training forward of the Gumbel-softmax estimator (the ablation of Sec. 7):
 * every pixel with p > 0 gets its extra sample, weighted by
 * sigma(lambda (ln(p / (1 - p)) + ln(u / (1 - u)))), lambda the inverse
 * temperature; the count map then exceeds B N (capacity for about N (1 + B)
 * samples).  Not with the systematic map. */
#define SPP_HOLDOUT_GUMBEL 2
/* the deterministic rounding of DASR (Sec. 4.1, Eq. kuz_fw, after Kuznetsov
 * et al. 2018), the ablation of Sec. 7: n_i = round(s_i) with halves going
 * up (floor(s_i) + [s_i - floor(s_i) >= 1/2], decided in FP64), no uniform
 * and no holdout weight (holdout_w = 1).  s_out then receives max(n_i, 1),
 * so that spp_splat_samples computes Eq. kuz_fw, L0_i = (sum_{j<n_i}
 * S_ij) / n_i and 0 without samples.  The same rule serves training and
 * test time.  Not with the systematic map. */
#define SPP_HOLDOUT_DASR 3

/* spp_params.flags */
#define SPP_FLAG_EXACT_FP64 1u /* evaluate every pixel on the FP64 path (no FP32 filter) */
/* Test of the bounded waits: scan tile 1 never publishes its prefix, so the
 * look-back waits of the later tiles run out; the call completes with
 * SPP_ERR_TIMEOUT in the status word and meaningless offsets. */
#define SPP_FLAG_TEST_STALL_TILE1 (1u << 31)

/* Sampling parameters (Sec. 3, Sec. 4.2-4.3). */
typedef struct spp_params {
    double budget;           /* B: mean samples per pixel of the frame, > 0 */
    double uniform_fraction; /* phi: part of the budget spread uniformly; the paper uses 1/8 */
    double lambda;           /* ramp temperature, >= 1; the paper uses 10 */
    uint64_t seed;           /* seed of the per-pixel uniforms u_i */
    uint32_t frame;          /* frame index t (selects the uniform stream) */
    int32_t holdout_mode;    /* SPP_HOLDOUT_RAMP, _HARD, _GUMBEL or _DASR */
    uint32_t flags;          /* SPP_FLAG_* */
    uint32_t reserved;       /* must be 0 */
} spp_params;

/* Tone-map parameters (Sec. 5): contrast alpha, saturation beta, exposure k,
 * shadow s in (0,1), highlight h in (0,1).  Defaults 1, 1, 0, 0.5, 0.5. */
typedef struct spp_tonemap {
    float alpha;
    float beta;
    float exposure;
    float shadow;
    float highlight;
} spp_tonemap;

/* ------------------------------------------------------------ utilities */
/* Message for an SPP_* code; never NULL. */
const char *spp_strerror(int code);

/* ABI version of this header (increases on incompatible change). */
int spp_abi_version(void);

/* Number of kernels this library has launched in this process (host-side
 * counter, incremented at every launch). */
uint64_t spp_launch_count(void);

/* Programmatic dependent launch of the plain path's kernels (sample map,
 * renderer stand-in, splat, pipelined reconstruction): when on (the
 * default), each may be scheduled while the kernel before it in the stream
 * is still running and waits on the device for that kernel's completion
 * before it touches memory, so launch latency and block start-up overlap the
 * previous kernel's tail.  Results are identical either way.  Process-wide;
 * spp_set_dependent_launch returns the previous setting. */
int spp_set_dependent_launch(int on);
int spp_get_dependent_launch(void);

/* Test of the bounded waits of the pipelined reconstruction: the next
 * launch of the pipelined kernel (spp_reconstruct_level, or a level of
 * spp_reconstruct_frame, whose width is a multiple of 4) issues no copies
 * for its tile number `tile` (tiles of 64 x 4 pixels, row-major), so the
 * waits for that tile run out after about 100 ms; that launch then records
 * SPP_ERR_TIMEOUT in its status word, the tiles after it in the same CTA
 * stay unwritten, and later calls are unaffected.  One-shot and
 * process-wide; -1 (the default) cancels.  SPP_ERR_ARG for tile < -1. */
int spp_test_stall_reconstruction(int tile);

/* Copies the device status word to the host (synchronises the stream) and
 * returns it (SPP_OK or an SPP_ERR_* code); SPP_ERR_CUDA if the copy fails. */
int spp_get_status(const int32_t *status, cudaStream_t stream);

/* Resets the device status word to SPP_OK (asynchronous). */
int spp_clear_status(int32_t *status, cudaStream_t stream);

/* ---------------------------------------------------- a1-a3: allocation */
/* Blue-noise dithering (Sec. 6.3 dithers the discretisation with blue
 * noise, after Ulichney's void-and-cluster method).  spp_blue_noise_mask
 * writes a T x T rank matrix (T a power of two in [4, 256], a permutation of
 * 0 .. T^2-1) to HOST memory `rank`: void-and-cluster on a torus with a
 * Gaussian filter of sigma 1.5 whose weights are the integers
 * round(2^20 exp(-r^2 / 4.5)), ties broken by the smallest index, the start
 * pattern of floor(T^2/10) pixels drawn by SplitMix64(seed).  SPP_ERR_ARG for
 * a bad T or a null pointer.  Upload the result to use it with
 * spp_alloc_sample_map_dithered. */
int spp_blue_noise_mask(int T, uint64_t seed, uint16_t *rank);

/* Workspace bytes spp_alloc_sample_map needs for a W x H frame. */
size_t spp_alloc_workspace_bytes(int W, int H);

/*
 * Turns a sampler density into an integer sample-count map and a sample list
 * (Sec. 3: 1/8 of the budget uniform, 7/8 by the spatial softmax of d;
 * Sec. 4.2: stochastic rounding; Sec. 4.3, Eq. relaxed_holdout and h_factor:
 * the relaxed holdout weight).
 *
 *   d            [H][W] FP32 sampler output, >= 0 (already exponentiated, so
 *                d_i / sum d is the softmax).  NaN, inf, negative values or an
 *                all-zero map set SPP_ERR_INPUT in *status; the outputs are
 *                then zero counts, s = 1, weights 1.
 *   p            sampling parameters (host pointer).
 *   counts       [H][W] int32 n_i, or NULL to skip.
 *   offsets      [H*W + 1] int32 exclusive scan of n; offsets[H*W] = T.  The
 *                samples of pixel i are slots offsets[i] .. offsets[i+1]-1,
 *                its extra (holdout) sample, if any, is the last of them.
 *   sample_pixel [capacity] int32 pixel index of every slot < min(T, capacity).
 *   capacity     number of slots sample_pixel (and the renderer's sample
 *                buffer) hold.  T > capacity sets SPP_ERR_CAPACITY.
 *   s_out        [H][W] FP32 density s_i = B phi + (1-phi) B N d_i / sum d.
 *   holdout_w    [H][W] FP32 weight of pixel i's last slot: the ramp weight
 *                H_i / S_i,last when the extra sample is taken, else 1.
 *   total        device int64 T (number of samples).
 *   status       device int32 status word.
 *   ws, ws_bytes workspace of at least spp_alloc_workspace_bytes(W, H).
 *
 * The count map is bit-exact to the FP64 definition: sum d is computed
 * exactly and rounded once to FP64, and s_i, floor(s_i), p_i and the test
 * u_i > 1 - p_i are decided as FP64 round-to-nearest operations (an FP32
 * filter settles the pixels whose decision is not close; the rest run in
 * FP64).  u_i = (bits >> 16) 2^-48 with bits the SplitMix64 mix of
 * key + (i+1) gamma, key = mix(seed + (frame+1) gamma).
 * Requires B * N + N < 2^31.
 */
int spp_alloc_sample_map(const float *d, int W, int H, const spp_params *p,
                         int32_t *counts, int32_t *offsets, int32_t *sample_pixel,
                         int64_t capacity, float *s_out, float *holdout_w, int64_t *total,
                         int32_t *status, void *ws, size_t ws_bytes, cudaStream_t stream);

/* spp_alloc_sample_map with the uniforms taken from a blue-noise mask
 * (device, uint16 [T][T], from spp_blue_noise_mask) tiled over the frame
 * instead of the counter-based white noise: for pixel (x, y) of frame
 * p->frame,
 *   u = ((rank[y mod T][x mod T] 2^(48-2k) + 2^(47-2k) + off) mod 2^48) 2^-48,
 *   T = 2^k, off = (frame G + (mix(seed) >> 16)) mod 2^48,
 * G = 0x9E3779B97F4A (the golden-ratio gamma's top 48 bits), mix the
 * SplitMix64 finaliser.  Within a tile the uniforms of a frame are the
 * stratified values (r + 1/2)/T^2 in blue-noise order, so a constant density
 * receives its budget to within one sample per tile; the golden-ratio step
 * moves each pixel's threshold from frame to frame.  Other arguments and
 * errors as spp_alloc_sample_map. */
int spp_alloc_sample_map_dithered(const float *d, int W, int H, const spp_params *p,
                                  const uint16_t *mask, int T, int32_t *counts, int32_t *offsets,
                                  int32_t *sample_pixel, int64_t capacity, float *s_out,
                                  float *holdout_w, int64_t *total, int32_t *status, void *ws,
                                  size_t ws_bytes, cudaStream_t stream);

/*
 * Allocation-free variant of spp_alloc_sample_map.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * while they run, such as an engine or plug-in host that owns the GPU memory
 * budget and forbids allocation inside its frame loop (cudaMalloc can
 * synchronise the device and take unbounded time).
 *
 * Same arguments and results as spp_alloc_sample_map, without the workspace:
 * the scratch lives in a library-owned static device array of 131,328 bytes,
 * which every GPU that loads the library keeps until the process exits.
 *   - Frames are limited to W*H <= 33,554,432 pixels (2^25); larger frames
 *     return SPP_ERR_WORKSPACE and enqueue nothing.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the one array and each call clears the part it uses
 *     before use.  Calls that overlap on the GPU (for example on two streams
 *     at once) race on it: issue them on one stream, one after the other.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.
 */
int spp_alloc_sample_map_static(const float *d, int W, int H, const spp_params *p,
                                int32_t *counts, int32_t *offsets, int32_t *sample_pixel,
                                int64_t capacity, float *s_out, float *holdout_w, int64_t *total,
                                int32_t *status, cudaStream_t stream);

/* ---------------------------------------------- a4: renderer stand-in */
/*
 * Stand-in for the path tracer, which the paper runs in Falcor (Sec. 3, Sec.
 * 6.3): sample k of pixel i is clean_i * exp(0.8 Z - 0.32), Z ~ N(0,1) by
 * Box-Muller from two SplitMix64 counters of (seed, frame, i, k).
 *
 *   clean        [3][H][W] FP32 clean image.
 *   offsets, sample_pixel, total   the sample list of spp_alloc_sample_map.
 *   capacity     slots in rgb; slots >= min(T, capacity) are not written.
 *   rgb          [capacity][4] FP32 (r, g, b, 0) per slot.
 */
int spp_render_synthetic(const float *clean, const int32_t *offsets, const int32_t *sample_pixel,
                         const int64_t *total, int64_t capacity, int W, int H, uint64_t seed,
                         uint32_t frame, float *rgb, cudaStream_t stream);

/* --------------------------------------------- a5: splat and pyramid */
/*
 * Normalised splat of Eq. stoch_rnoisy, L0_i = (sum_{k<floor s_i} S_ik + H_i)/s_i,
 * and the average-pool pyramid of Eq. app-pyramid, L^l = 4^-l sum over the
 * 2^l x 2^l block.  Each pixel gathers its own slots (the sample list is
 * ordered by pixel), so no atomics are used and the result is deterministic.
 *
 *   offsets      [H*W + 1] from spp_alloc_sample_map.
 *   rgb          [capacity][4] samples (spp_render_synthetic layout).
 *   s, holdout_w [H][W] from spp_alloc_sample_map.
 *   capacity     slots in rgb; reads never go past it.
 *   layers       host array of L device pointers, layers[l] = [3][H>>l][W>>l].
 */
int spp_splat_samples(const int32_t *offsets, const float *rgb, const float *s,
                      const float *holdout_w, int64_t capacity, int W, int H, int L,
                      float *const *layers, cudaStream_t stream);

/* ---------------------------------------- a6-a9: reconstruction, tau */
/* Workspace bytes of spp_reconstruct_frame (the denoised levels 1..L-1 and
 * the warped previous frame). */
size_t spp_reconstruct_workspace_bytes(int W, int H, int L);

/* Tone map of a whole image (Sec. 5, the epilogue of the full-resolution
 * reconstruction applied on its own): ldr [3][H][W] = sRGB(tau(x)) of hdr
 * [3][H][W], for reference images and the recurrent network input. */
int spp_tonemap_image(const float *hdr, int W, int H, const spp_tonemap *tm, float *ldr,
                      cudaStream_t stream);

/*
 * W_t L_{t-1}: the previous HDR output warped along the motion vectors
 * (App. A, Eq. app-recon-full; Sec. 6.1).  warped(x, y) is the bilinear sample
 * of prev_hdr at (x + mv_x, y + mv_y), pixel centres at integer coordinates,
 * the position clamped to [0, W-1] x [0, H-1].
 *   prev_hdr [3][H][W]; mv [2][H][W] in pixels, current -> previous;
 *   warped   [3][H][W] output.
 */
int spp_warp_previous(const float *prev_hdr, const float *mv, int W, int H, float *warped,
                      cudaStream_t stream);

/*
 * One level of the coarse-to-fine reconstruction (Appendix A):
 * Eq. app-recon-coarse when coarse == NULL, Eq. app-recon-mid otherwise, and
 * Eq. app-recon-full when warped_prev != NULL.  The joint softmax (Eq.
 * app-softmax-mid, app-softmax-full) spans the 25 denoise logits, the 4
 * upsampling logits when coarse != NULL, and the 25 temporal logits when
 * warped_prev != NULL and mask is 0 at the pixel.
 *
 *   noisy     [3][Hl][Wl] noisy level L^l.
 *   logits    [C][Hl][Wl]: channels 0..24 denoise tap (i,j) at (j+2)*5+(i+2);
 *             25..28 upsampling tap (i,j) at 25+2j+i; 29..53 temporal taps.
 *             C >= 25, >= 29 with coarse, == 54 with prev_hdr.
 *   coarse    [3][Hl/2][Wl/2] denoised L-hat^{l+1}, or NULL at the coarsest level.
 *   warped_prev [3][Hl][Wl] W_t L_{t-1} from spp_warp_previous, or NULL (no
 *             temporal term).
 *   mask      [Hl][Wl] uint8, nonzero = disoccluded (drops the temporal
 *             logits), or NULL.
 *   tm        tone map for out_ldr, or NULL for the defaults.
 *   out       [3][Hl][Wl] reconstructed HDR level.
 *   out_ldr   [3][Hl][Wl] sRGB(tau(...)) of out (Sec. 5), or NULL.
 *   status    device int32 status word, or NULL; a bounded wait of the
 *             pipelined kernel that gave up records SPP_ERR_TIMEOUT there.
 * Borders clamp to the edge; the upsampling taps read floor((x+i)/2),
 * floor((y+j)/2) of the coarser level as printed in Eq. app-upsample.
 * Levels whose width is a multiple of 4 run a persistent kernel fed by bulk
 * tensor copies (TMA) through a multi-stage shared-memory pipeline; other
 * widths run a direct kernel.  Both compute the same values.
 */
int spp_reconstruct_level(const float *noisy, const float *logits, int C, const float *coarse,
                          const float *warped_prev, const uint8_t *mask, int Wl, int Hl,
                          const spp_tonemap *tm, float *out, float *out_ldr, int32_t *status,
                          cudaStream_t stream);

/*
 * The whole reconstruction: levels L-1 .. 1 into the workspace, then level 0
 * with the temporal term and the tone map (Appendix A; Sec. 5).
 *   layers   host array of L pointers to the noisy pyramid (spp_splat_samples).
 *   logits   host array of L pointers: logits[L-1] has 25 channels, logits[l]
 *            for 0 < l < L-1 has 29, logits[0] has C0 (29, or 54 with temporal).
 *   C0       channels of logits[0]: 29 or 54.  prev_hdr != NULL needs 54.
 *   prev_hdr [3][H][W] previous HDR output or NULL; mv [2][H][W] with it.
 *            The frame call warps it (spp_warp_previous) into the workspace.
 *   L        pyramid levels, 2..5.
 *   out_hdr  [3][H][W]; out_ldr [3][H][W] or NULL.
 *   status   device int32 status word, or NULL (see spp_reconstruct_level).
 */
int spp_reconstruct_frame(const float *const *layers, const float *const *logits, int C0,
                          const float *prev_hdr, const float *mv, const uint8_t *mask, int W,
                          int H, int L, const spp_tonemap *tm, float *out_hdr, float *out_ldr,
                          void *ws, size_t ws_bytes, int32_t *status, cudaStream_t stream);

/* ------------------------------------------------------ a11: backward */
/*
 * Gradients of the path, for training the sampler and the kernel predictor
 * end to end (Sec. 4.3, Sec. 5, Sec. 6.3).  Each call maps the gradient of
 * the loss with respect to a step's output to its inputs' gradients.  Unless
 * stated otherwise a gradient output is ACCUMULATED (+=): the caller zeroes
 * it, and several calls may add into one buffer.  Every gradient is summed
 * in a fixed order (each output element has one writer), so the results are
 * the same from run to run, except spp_warp_previous_backward's, which
 * scatters with floating-point atomics.
 */

/* Reconstruction level (Appendix A) given dLoss/d out (grad_out, [3][Hl][Wl]).
 * Recomputes each pixel's joint softmax from its logits.
 *   grad_logits [C][Hl][Wl], OVERWRITTEN: w_k (q_k - sum_j w_j q_j) with
 *               q_k = sum_c grad_out_c v_kc; 0 for channels without a kernel
 *               (and for the temporal channels of disoccluded pixels).
 *   grad_noisy  [3][Hl][Wl], grad_coarse [3][Hl/2][Wl/2], grad_warped
 *               [3][Hl][Wl]: += w_k grad_out at each tap's source pixel
 *               (clamp-to-edge transposed); each may be NULL.
 * Other arguments as in spp_reconstruct_level. */
int spp_reconstruct_level_backward(const float *noisy, const float *logits, int C,
                                   const float *coarse, const float *warped_prev,
                                   const uint8_t *mask, int Wl, int Hl, const float *grad_out,
                                   float *grad_logits, float *grad_noisy, float *grad_coarse,
                                   float *grad_warped, cudaStream_t stream);

/* W_t backward: grad_prev [3][H][W] += the bilinear weights of every pixel
 * applied to grad_warped (the transpose of spp_warp_previous). */
int spp_warp_previous_backward(const float *mv, int W, int H, const float *grad_warped,
                               float *grad_prev, cudaStream_t stream);

/* Tone-map backward (Sec. 5): grad_hdr [3][H][W] += d sRGB(tau(x)) / d hdr
 * applied to grad_ldr; pixels at the 2^-24 floor get no gradient. */
int spp_tonemap_backward(const float *hdr, int W, int H, const spp_tonemap *tm,
                         const float *grad_ldr, float *grad_hdr, cudaStream_t stream);

/* Spatial loss of Eq. loss_spatial with m = 1: *loss (device float) =
 * mean |ldr - ref| over n values; grad_ldr (OVERWRITTEN, or NULL) =
 * sign(ldr - ref) / n. */
int spp_l1_loss(const float *ldr, const float *ref, int64_t n, float *loss, float *grad_ldr,
                cudaStream_t stream);

/* Combined training loss of Sec. 6.3 (Eq. loss_spatial with the mask m = 1,
 * Eq. loss_temporal, Eq. loss_combined) over n elements of tone-mapped sRGB:
 *   *loss (device float, OVERWRITTEN) = mean of max(wt |dI - dI_ref|, ws |I - I_ref|)
 * with dI = ldr - prev_warped and dI_ref = ref - ref_prev_warped (the previous
 * output and reference, warped to this frame, e.g. by spp_warp_previous),
 * wt = temporal_weight, ws = spatial_weight (the paper: 1.25 and 1; ws = 0
 * gives the temporal error alone); the maximum is taken per element, ties go
 * to the spatial term.  grad_ldr (nullable, OVERWRITTEN) = d loss / d ldr
 * with the previous frame held constant. */
int spp_combined_loss(const float *ldr, const float *ref, const float *prev_warped,
                      const float *ref_prev_warped, int64_t n, float temporal_weight,
                      float spatial_weight, float *loss, float *grad_ldr, cudaStream_t stream);

/* Evaluation metric: *mse (device double, OVERWRITTEN) = mean over the n
 * elements of (a - b)^2, accumulated in FP64.  PSNR = -10 log10(mse) for
 * images in [0, 1]. */
int spp_mse(const float *a, const float *b, int64_t n, double *mse, cudaStream_t stream);

/* Pyramid backward (Eq. app-pyramid): grad_L0 [3][H][W] += sum over levels
 * l >= 1 of 4^-l grad_layers[l] at the pixel's coarse cell (grad_layers[0]
 * is not read). */
int spp_pyramid_backward(const float *const *grad_layers, int W, int H, int L, float *grad_L0,
                         cudaStream_t stream);

/* Splat backward (Eq. stoch_rnoisy, Eq. relaxed_holdout) with respect to the
 * density s, the discrete choices held fixed:
 *   grad_s_i = sum_c g_ic (-L0_ic / s_i)
 *            + [extra, ramp in its linear part] sum_c g_ic S_i,last,c / s_i
 *              * h lambda (1 - u_i) / p_i^2
 * grad_s [H][W] is OVERWRITTEN.  offsets, counts, rgb, s come from the
 * forward calls; layer0 is L0 and grad_layer0 dLoss/dL0; p the sampling
 * parameters of the forward call (u_i is recomputed from seed and frame). */
int spp_splat_backward(const int32_t *offsets, const int32_t *counts, const float *rgb,
                       const float *s, const float *layer0, const float *grad_layer0,
                       int64_t capacity, int W, int H, const spp_params *p, float *grad_s,
                       cudaStream_t stream);

/* Workspace bytes of spp_density_backward. */
size_t spp_density_backward_workspace_bytes(void);

/* Density backward (Sec. 3): with s = phi B + (1-phi) B N d / sum d and
 * d = exp(z - max z) the sampler's softmax, grad_z (OVERWRITTEN) =
 * (1-phi) B N pi (grad_s - sum_i pi_i grad_s_i), pi = d / sum d. */
int spp_density_backward(const float *d, int64_t N, double budget, double uniform_fraction,
                         const float *grad_s, float *grad_z, void *ws, size_t ws_bytes,
                         cudaStream_t stream);


/* --------------------------------------------- a10: learned predictor */
/*
 * The network that predicts the sampling density and the per-level kernel
 * logits from G-buffers and the previous output (Sec. 3, Sec. 6.3,
 * Appendix A): a U-Net of 3x3 convolutions (zero padding, bias), ReLU after
 * the hidden layers, 2x2 average pooling on the way down, nearest
 * upsampling and channel concatenation on the way up.  The paper prints no
 * layer table; this library's reading, in parameter order
 * (spp_unet_layer):
 *    0 e0a  12->32            1 e0b 32->32       level 0 (full resolution)
 *    2 e1a  32->64  (input: 2x2 pool of e0b)      3 e1b 64->64    level 1
 *    4 e2a  64->128 (input: 2x2 pool of e1b)      5 e2b 128->128  level 2
 *    6 h2  128->25  level-2 kernel logits (linear)
 *    7 d1a 192->64  (input: concat [e1b, upsampled e2b])  8 d1b 64->64
 *    9 h1   64->29  level-1 kernel logits (linear)
 *   10 d0a  96->32  (input: concat [e0b, upsampled d1b]) 11 d0b 32->32
 *   12 h0   32->55  level-0 kernel logits (channels 0..53: kd 25, ku 4,
 *                   kt 25) and the density logit z (channel 54)
 * Parameters theta: FP32, for each layer in order the weights
 * [cout][cin][3][3] followed by the bias [cout].
 *
 * Precision: BF16 weights and activations (round to nearest even), FP32
 * accumulation on the tcgen05 tensor cores, FP32 biases and logits.
 * Activations are stored NHWC (channels innermost) in BF16; the images the
 * reconstruction reads (logits, density) are planar FP32.
 */
#define SPP_UNET_LAYERS 13
#define SPP_UNET_FEATURES 12
#define SPP_UNET_DENSITY_CHANNEL 54

/* Shape of layer i (0..12): input and output channels, 1 if ReLU follows.
 * SPP_ERR_ARG for i out of range or a null pointer. */
int spp_unet_layer(int i, int *cin, int *cout, int *relu);

/* Number of FP32 parameters in theta (535565). */
int64_t spp_unet_param_count(void);

/* Bytes of the packed parameter blob: BF16 weights in the tensor-core
 * operand layout and FP32 biases of every layer, plus, when with_backward
 * is non-zero, the flipped and transposed weights the data gradient uses. */
size_t spp_unet_packed_bytes(int with_backward);

/* Packs theta (device FP32, spp_unet_param_count values) into `packed`
 * (device, spp_unet_packed_bytes(with_backward) bytes, 256-byte aligned).
 * Re-run after every change of theta. */
int spp_unet_pack(const float *theta, int with_backward, void *packed, size_t packed_bytes,
                  cudaStream_t stream);

/* Network input of one W x H frame (Sec. 6.3 G-buffer inputs plus the
 * previous output of Sec. 3): in12 [12][H][W] = albedo [3], normal [3],
 * ln(depth)/ln(100) [1] (depth [H][W] > 0), motion / 8 px [2] (mv
 * [2][H][W]), previous LDR output warped to this frame [3] (prev_ldr; NULL
 * gives zeros, the first frame). */
int spp_assemble_features(const float *albedo, const float *normal, const float *depth,
                          const float *mv, const float *prev_ldr, int W, int H, float *in12,
                          cudaStream_t stream);

/* Workspace bytes of spp_predict_density_and_kernels for B frames of
 * W x H (the activations of every layer; the backward reads them). */
size_t spp_predict_workspace_bytes(int B, int W, int H);

/* Forward pass of the predictor on B frames (W, H divisible by 4):
 *   in12     [B][12][H][W] FP32 input features
 *   density  [B][H][W] FP32: d = exp(z - max z) per frame, the unnormalised
 *            spatial softmax (Sec. 3) that spp_alloc_sample_map normalises
 *   logits0  [B][55][H][W] FP32: planes 0..53 are the level-0 kernel logits
 *            (the first 29 planes are the logits without the temporal
 *            term), plane 54 the density logit z
 *   logits1  [B][29][H/2][W/2], logits2 [B][25][H/4][W/4] FP32
 * packed comes from spp_unet_pack; ws keeps the activations for the
 * backward.  Device-side errors (a tensor-core pipeline wait that gave up)
 * land in *status. */
int spp_predict_density_and_kernels(const void *packed, const float *in12, int B, int W, int H,
                                    float *density, float *logits0, float *logits1,
                                    float *logits2, void *ws, size_t ws_bytes, int32_t *status,
                                    cudaStream_t stream);

/* Single 3x3 convolution layers on the tensor cores (the building block of
 * the predictor, exposed for testing and reuse).  Tensors are BF16 (as
 * uint16_t bit patterns) in NHWC layout [B][H][W][C]; weights w
 * [cout][cin][3][3] and bias [cout] are FP32 and are packed into ws.
 * Channel counts of BF16 tensors must be multiples of 8; the output channel
 * count of a call (cout for the forward, cin for the data gradient) must be
 * one of 16, 32, 64, 96, 128, 192. */
size_t spp_conv3x3_workspace_bytes(int cin, int cout);

/* y = conv3x3(x, w) + bias, then max(., 0) if relu. */
int spp_conv3x3_forward(const uint16_t *x, int B, int W, int H, int cin, int cout, const float *w,
                        const float *bias, int relu, uint16_t *y, void *ws, size_t ws_bytes,
                        int32_t *status, cudaStream_t stream);

/* Data gradient: gx = conv3x3^T(g) (g [B][H][W][cout], gx [B][H][W][cin]),
 * multiplied by (act > 0) elementwise when act ([B][H][W][cin]) is given
 * (the ReLU of the layer that produced the input). */
int spp_conv3x3_backward_data(const uint16_t *g, int B, int W, int H, int cin, int cout,
                              const float *w, const uint16_t *act, uint16_t *gx, void *ws,
                              size_t ws_bytes, int32_t *status, cudaStream_t stream);


/* Weight gradient of a 3x3 layer: gw [cout][cin][3][3] = sum over pixels
 * of g (x) the shifted x, gb [cout] = sum over pixels of g (both FP32,
 * OVERWRITTEN; gb may be NULL).  x [B][H][W][cin] and g [B][H][W][cout] are
 * BF16 NHWC (cin, cout multiples of 8, cout <= 128).  The partial sums of
 * the pixel splits are added in a fixed order, so the result is
 * deterministic. */
size_t spp_conv3x3_backward_weights_workspace_bytes(int B, int W, int H, int cin, int cout);
int spp_conv3x3_backward_weights(const uint16_t *x, const uint16_t *g, int B, int W, int H,
                                 int cin, int cout, float *gw, float *gb, void *ws,
                                 size_t ws_bytes, int32_t *status, cudaStream_t stream);

/* ------------------------------------- a11: training the predictor */
/* Workspace bytes of spp_unet_backward. */
size_t spp_unet_backward_workspace_bytes(int B, int W, int H);

/* Backward of spp_predict_density_and_kernels (Sec. 6.3 training): from the
 * gradients of the loss with respect to its outputs,
 *   grad_logits0 [B][55][H][W] (planes 0..53 the level-0 kernel logits,
 *                plane 54 the density logit z, e.g. from
 *                spp_density_backward),
 *   grad_logits1 [B][29][H/2][W/2], grad_logits2 [B][25][H/4][W/4],
 * computes grad_theta (FP32, the layout of theta, OVERWRITTEN).  packed must
 * come from spp_unet_pack(theta, with_backward = 1); fwd_ws is the
 * workspace of the forward call on the same in12 (its activations are read,
 * not recomputed).  Gradients between layers are BF16 NHWC; every
 * contraction runs on the tensor cores with FP32 accumulation. */
int spp_unet_backward(const void *packed, const float *in12, int B, int W, int H,
                      const void *fwd_ws, size_t fwd_ws_bytes, const float *grad_logits0,
                      const float *grad_logits1, const float *grad_logits2, float *grad_theta,
                      void *ws, size_t ws_bytes, int32_t *status, cudaStream_t stream);

/* One AdamW step (Loshchilov & Hutter, decoupled weight decay) on n FP32
 * parameters, step >= 1 (bias correction 1 - beta^step):
 *   g = grad_scale * grad; m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 *   theta -= lr (m / (1-b1^step) / (sqrt(v / (1-b2^step)) + eps) + wd theta).
 * m and v start at zero. */
int spp_adamw_step(float *theta, const float *grad, float *m, float *v, int64_t n, int step,
                   float lr, float beta1, float beta2, float eps, float weight_decay,
                   float grad_scale, cudaStream_t stream);

/* ------------------------- f1: two-stage pipeline (sampler + denoiser) */
/*
 * The paper's full pipeline (Sec. 3, Sec. 6.2 "Learned Demodulation",
 * Sec. 6.3): a sampler network predicts the density before rendering; after
 * rendering a denoiser network sees the noisy radiance, the sample maps, the
 * G-buffer, the previous HDR output and latent features, and predicts the
 * gather-kernel logits, a 3-channel demodulation map and the latents that
 * both networks read (warped) in the next frame.  The paper prints neither
 * layer tables nor input encodings; this library's reading:
 *
 * Networks (same U-Net trunk as the joint predictor above, layer slots
 * 0..12 of spp_unet_layer; a network without h1 / h2 leaves those slots
 * empty, cout = 0, and has no parameters for them):
 *   SPP_NET_JOINT     12 inputs; h0 55 (54 logits + density logit), h1 29, h2 25
 *   SPP_NET_SAMPLER   19 inputs: the 12 joint features, then the 7 warped
 *                     latents; h0 = 1 (density logit z)
 *   SPP_NET_DENOISER  24 inputs: ln(1+L^0) [3], ln(1+s), ln(1+n), albedo [3],
 *                     normal [3], ln(depth)/ln(100), motion/8 [2],
 *                     ln(1 + W_t L_{t-1}) [3], warped latents [7];
 *                     h0 = 64 planes: 54 kernel logits, 3 raw demodulation
 *                     channels c (planes 54..56), 7 raw latents (57..63);
 *                     h1 29, h2 25
 * Demodulation map m = exp(clamp(c, -8, 8)); latents passed on = tanh of
 * their raw planes.  Frame with demodulation:
 *   hdr = m * R(pyramid(L^0 / m), W_t L_{t-1} / m, kernel logits)
 * where R is the gather pyramid (spp_reconstruct_level, levels L-1 .. 0).
 */
#define SPP_NET_JOINT 0
#define SPP_NET_SAMPLER 1
#define SPP_NET_DENOISER 2
#define SPP_LATENT_CHANNELS 7
#define SPP_DEMOD_PLANE 54
#define SPP_LATENT_PLANE 57

/* Input channels and head widths (0 = absent) of network `net`. */
int spp_net_spec(int net, int *cin, int *head0, int *head1, int *head2);
/* Shape of layer slot i (0..12) of network `net` (cout 0: absent head). */
int spp_net_layer(int net, int i, int *cin, int *cout, int *relu);
/* FP32 parameters of network `net` (-1 for an unknown net). */
int64_t spp_net_param_count(int net);
/* Packed blob bytes / packing, as spp_unet_packed_bytes / spp_unet_pack. */
size_t spp_net_packed_bytes(int net, int with_backward);
int spp_net_pack(int net, const float *theta, int with_backward, void *packed,
                 size_t packed_bytes, cudaStream_t stream);
/* Forward workspace bytes (activations kept for the backward). */
size_t spp_net_workspace_bytes(int net, int B, int W, int H);
/* Forward on B frames (W, H divisible by 4, else SPP_ERR_SHAPE): in
 * [B][cin][H][W] FP32; head0 [B][h0][H][W], head1 [B][h1][H/2][W/2], head2
 * [B][h2][H/4][W/4] FP32 planar (NULL allowed for an absent head, required
 * for a present one: SPP_ERR_ARG).  packed and ws 256-byte aligned
 * (SPP_ERR_ALIGN); ws at least spp_net_workspace_bytes (SPP_ERR_WORKSPACE);
 * unknown net: SPP_ERR_ARG. */
int spp_net_forward(int net, const void *packed, const float *in, int B, int W, int H,
                    float *head0, float *head1, float *head2, void *ws, size_t ws_bytes,
                    int32_t *status, cudaStream_t stream);
/* Where the forward keeps its BF16 NHWC copy of the input inside ws: byte
 * offset and channels (the input padded to 16 or 32; image b starts at
 * offset + b H W channels 2 bytes).  spp_assemble_sampler_input /
 * spp_assemble_denoiser_input write it there directly, and
 * spp_net_forward_prepared then runs the network without the FP32 input
 * (the same results as spp_net_forward on the FP32 features; the same
 * argument checks).  spp_net_input_layout: SPP_ERR_ARG for an unknown net,
 * a negative size or a NULL output pointer. */
int spp_net_input_layout(int net, int B, int W, int H, size_t *offset, int *channels);
int spp_net_forward_prepared(int net, const void *packed, int B, int W, int H, float *head0,
                             float *head1, float *head2, void *ws, size_t ws_bytes,
                             int32_t *status, cudaStream_t stream);
size_t spp_net_backward_workspace_bytes(int net, int B, int W, int H);
/* Backward of spp_net_forward: grad_theta (OVERWRITTEN) from the head
 * gradients (same shapes as the heads); if grad_in is not NULL also the
 * gradient with respect to the input, [B][cin][H][W] FP32 (OVERWRITTEN; the
 * BF16 rounding of the input counts as the identity).  fwd_ws: the
 * workspace of the forward call. */
int spp_net_backward(int net, const void *packed, int B, int W, int H, const void *fwd_ws,
                     size_t fwd_ws_bytes, const float *grad_head0, const float *grad_head1,
                     const float *grad_head2, float *grad_theta, float *grad_in, void *ws,
                     size_t ws_bytes, int32_t *status, cudaStream_t stream);

/* Unnormalised spatial softmax of a density logit plane per frame:
 * density[b][i] = exp(z[b * batch_stride + i] - max_i z[b * batch_stride + i])
 * (Sec. 3); ws holds B words. */
size_t spp_density_softmax_workspace_bytes(int B);
int spp_density_softmax(const float *z, int B, int W, int H, int64_t batch_stride,
                        float *density, void *ws, size_t ws_bytes, cudaStream_t stream);

/* Latents of frame t-1 for frame t: out[k] = W_t tanh(raw[k]) for the 7
 * raw latent planes of the previous denoiser (raw [7][H][W], usually head0
 * + 57 planes), bilinear along mv like spp_warp_previous. */
int spp_warp_latent(const float *raw, const float *mv, int W, int H, float *out,
                    cudaStream_t stream);

/* The same in two steps, each source value's tanh taken once: out [7][H][W]
 * = tanh(raw) (spp_latent_tanh), then W_t of C planes along mv
 * (spp_warp_channels, the bilinear warp of spp_warp_previous on every
 * plane); spp_warp_channels(spp_latent_tanh(raw)) = spp_warp_latent(raw). */
int spp_latent_tanh(const float *raw, int W, int H, float *out, cudaStream_t stream);
int spp_warp_channels(const float *src, int C, const float *mv, int W, int H, float *out,
                      cudaStream_t stream);

/* Sampler input in19 [19][H][W]: the 12 channels of spp_assemble_features,
 * then warped_latent [7][H][W] (NULL: zeros, the first frame). */
int spp_assemble_sampler_features(const float *albedo, const float *normal, const float *depth,
                                  const float *mv, const float *warped_prev_ldr,
                                  const float *warped_latent, int W, int H, float *in19,
                                  cudaStream_t stream);

/* Denoiser input in24 [24][H][W] from the splatted radiance L0 [3][H][W],
 * the sample map s [H][W] and counts [H][W] (spp_alloc_sample_map), the
 * G-buffer, mv, the previous HDR output warped to this frame
 * (warped_prev_hdr [3][H][W], NULL: zeros) and the warped latents (NULL:
 * zeros), in the channel order given above. */
int spp_assemble_denoiser_features(const float *L0, const float *s, const int32_t *counts,
                                   const float *albedo, const float *normal, const float *depth,
                                   const float *mv, const float *warped_prev_hdr,
                                   const float *warped_latent, int W, int H, float *in24,
                                   cudaStream_t stream);

/* The same inputs written straight as the networks' BF16 NHWC input copy of
 * one image, [H][W][32] (x_nhwc32: inside the forward workspace, see
 * spp_net_input_layout; values rounded to nearest even from the FP32 values
 * above, channels 19 / 24 .. 31 zero). */
int spp_assemble_sampler_input(const float *albedo, const float *normal, const float *depth,
                               const float *mv, const float *warped_prev_ldr,
                               const float *warped_latent, int W, int H, uint16_t *x_nhwc32,
                               cudaStream_t stream);
int spp_assemble_denoiser_input(const float *L0, const float *s, const int32_t *counts,
                                const float *albedo, const float *normal, const float *depth,
                                const float *mv, const float *warped_prev_hdr,
                                const float *warped_latent, int W, int H, uint16_t *x_nhwc32,
                                cudaStream_t stream);

/* Adds the gradient reaching L0 and s through the denoiser input:
 * grad_L0 += grad_in24[0..2] / (1 + L0), grad_s += grad_in24[3] / (1 + s);
 * either output may be NULL (skipped), so that the L0 part can be added
 * before spp_splat_backward (which overwrites grad_s) and the s part after. */
int spp_denoiser_features_backward(const float *L0, const float *s, const float *grad_in24,
                                   int W, int H, float *grad_L0, float *grad_s,
                                   cudaStream_t stream);

/* Demodulation (Sec. 6.2): m = exp(clamp(c, -8, 8)) ([3][H][W], written to
 * m), layers[0] = L0 / m and layers[l] (l < L) the 2^l x 2^l block means of
 * layers[0] (Eq. app-pyramid); if warped is not NULL, warped_out = warped /
 * m.  W, H divisible by 2^(L-1), 1 <= L <= 5. */
int spp_demodulate(const float *L0, const float *c, const float *warped, int W, int H, int L,
                   float *m, float *const *layers, float *warped_out, cudaStream_t stream);

/* Remodulation and tone map: out_hdr = m * R ([3][H][W]), out_ldr =
 * tau-sRGB of out_hdr (tm as spp_reconstruct_level; out_ldr may be NULL). */
int spp_remodulate_tonemap(const float *R, const float *m, int W, int H, const spp_tonemap *tm,
                           float *out_hdr, float *out_ldr, cudaStream_t stream);

/* Backward of the remodulation into the reconstruction: grad_R = grad_out * m. */
int spp_remodulate_backward(const float *grad_out, const float *m, int W, int H, float *grad_R,
                            cudaStream_t stream);

/* Backward of the demodulation: from grad_out (w.r.t. out_hdr), grad_L0d
 * (w.r.t. layers[0], after spp_pyramid_backward folded the coarser levels
 * in) and grad_Wd (w.r.t. warped_out; NULL with Wd NULL), writes
 *   grad_L0 = grad_L0d / m
 *   grad_c  = (grad_out out_hdr - grad_L0d L0d - grad_Wd Wd) [|c| < 8]
 * (both OVERWRITTEN). */
int spp_demodulate_backward(const float *out_hdr, const float *grad_out, const float *L0d,
                            const float *grad_L0d, const float *Wd, const float *grad_Wd,
                            const float *c, const float *m, int W, int H, float *grad_L0,
                            float *grad_c, cudaStream_t stream);

/* ------------------------------------------ f4: variants of the pipeline */
/* Systematic (exact-integer-total) sample map: the reading of the budget of
 * Sec. 3 in which the realised total is fixed to within one sample.  The
 * pixels' intervals of length s_i (the same s_i as spp_alloc_sample_map) are
 * laid end to end from a frame offset U and every pixel receives the
 * integers its interval covers; in 32.32 fixed point (exact, independent of
 * the summation order):
 *   q_i = s_i 2^32 rounded to nearest even, P_i = q_0 + ... + q_i,
 *   offsets_i = (P_{i-1} + U) >> 32, n_i = offsets_{i+1} - offsets_i,
 *   T = (P_{N-1} + U) >> 32  (|T - B N| < 1 + N 2^-32),
 * U = the top 32 bits of element 2^62 of the (seed, frame) stream.  n_i is
 * floor(q_i 2^-32) plus one extra sample iff a_i + p_i >= 1 with a_i the
 * fractional position (P_{i-1} + U) mod 2^32 and p_i = q_i mod 2^32 (both
 * times 2^-32): the stochastic test of Sec. 4.2 at u = a_i; its holdout
 * weight is the ramp of Sec. 4.3 at u = a_i (1 in hard mode).  Arguments,
 * outputs and workspace as spp_alloc_sample_map (SPP_FLAG_TEST_STALL_TILE1
 * is rejected: this map has no waits between blocks). */
int spp_alloc_sample_map_systematic(const float *d, int W, int H, const spp_params *p,
                                    int32_t *counts, int32_t *offsets, int32_t *sample_pixel,
                                    int64_t capacity, float *s_out, float *holdout_w,
                                    int64_t *total, int32_t *status, void *ws, size_t ws_bytes,
                                    cudaStream_t stream);

/* Gradient estimators of the discretisation (the ablation of Sec. 7):
 * dLoss/ds of the splat (grad_s, OVERWRITTEN) with L^0 = (sum_{k<f} S_k +
 * e w S_f) / s, f = floor(s), p = s - f:
 *   SPP_ESTIMATOR_RELAXED           the relaxed ramp of Sec. 4.3, exactly
 *                                   spp_splat_backward
 *   SPP_ESTIMATOR_STRAIGHT_THROUGH  forward with SPP_HOLDOUT_HARD; de/dp := 1,
 *                                   so sum_c g_c (S_f,c - L^0_c) / s on every
 *                                   pixel with p > 0, S_f the traced extra
 *                                   sample, or, where the forward traced none,
 *                                   the renderer stand-in's sample of slot f
 *                                   (clean and render_seed as given to
 *                                   spp_render_synthetic, frame p->frame)
 *   SPP_ESTIMATOR_GUMBEL            forward with SPP_HOLDOUT_GUMBEL; dw/dp =
 *                                   lambda w (1 - w) / (p (1 - p)) with w =
 *                                   holdout_w of the forward
 *   SPP_ESTIMATOR_DASR              forward with SPP_HOLDOUT_DASR (Sec. 4.1);
 *                                   the surrogate of Eq. kuz_grad,
 *                                   sum_c g_c (ref_c - L^0_c) / n where
 *                                   n = counts_i >= 1, sum_c g_c ref_c where
 *                                   n = 0, with ref ([3][H][W], passed as
 *                                   `clean`) the reference radiance L^ref;
 *                                   reads counts, layer0, grad_layer0 and
 *                                   clean only
 * Other arguments as spp_splat_backward; clean is read by the
 * straight-through and DASR estimators only. */
#define SPP_ESTIMATOR_RELAXED 0
#define SPP_ESTIMATOR_STRAIGHT_THROUGH 1
#define SPP_ESTIMATOR_GUMBEL 2
#define SPP_ESTIMATOR_DASR 3
int spp_splat_backward_estimator(const int32_t *offsets, const int32_t *counts, const float *rgb,
                                 const float *s, const float *layer0, const float *grad_layer0,
                                 const float *holdout_w, int64_t capacity, int W, int H,
                                 const spp_params *p, int estimator, const float *clean,
                                 uint64_t render_seed, float *grad_s, cudaStream_t stream);

/* Low-resolution density map (the ablation of Sec. 7 that samples from a
 * density at a quarter of the pixels): out = P d, every factor x factor
 * block (factor 1, 2, 4 or 8 dividing W and H) replaced by its mean, summed
 * in FP32 as a pairwise tree (each row of the block: adjacent pairs, then
 * pairs of pairs; then the row sums, top to bottom) and scaled by
 * 1/factor^2.  P is a symmetric projection that keeps the sum, so the same
 * call maps the gradient with respect to out (grad_s of the allocation) to
 * the gradient with respect to d before spp_density_backward.  out may
 * equal d. */
int spp_density_lowres(const float *d, int W, int H, int factor, float *out,
                       cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SPP_H */
