// a6-a9: gather-pyramid reconstruction (Appendix A of arXiv 2602.08642) with
// the temporal term over the bilinearly reprojected previous output and the
// filmic tone map + sRGB epilogue (Sec. 5).
//
// One launch per pyramid level.  Levels whose row pitch is a multiple of 16
// bytes run the TMA-pipelined persistent kernel (reconstruct_tma.cu); the
// others run the direct kernel below.  In the direct kernel a block owns a
// 32 x 8 pixel tile: it stages the noisy level's tile plus a 2-pixel halo in
// shared memory and, at full resolution, the warped previous frame
// W_t L_{t-1} on the same halo (each halo pixel warped with its own motion
// vector), so that the 5 x 5 gathers read shared memory.  The per-pixel
// logits are read once, coalesced along x, and the joint softmax is evaluated
// in registers.
#include <algorithm>

#include "recon_common.cuh"

namespace spp {
namespace {

constexpr int kTX = 32;
constexpr int kTY = 8;
constexpr int kHalo = 2;
constexpr int kHX = kTX + 2 * kHalo;
constexpr int kHY = kTY + 2 * kHalo;

template <bool UP, bool TEMP, bool TONE>
__global__ void __launch_bounds__(kTX *kTY, 2)
recon_kernel(const float *__restrict__ noisy, const float *__restrict__ logits,
             const float *__restrict__ coarse, const float *__restrict__ warped,
             const uint8_t *__restrict__ mask, int Wl, int Hl, float *__restrict__ out,
             float *__restrict__ out_ldr, ToneArgs tm) {
    static_assert(!TEMP || UP, "the temporal term lives at full resolution, below a coarser level");
    constexpr int kSpatial = 25 + (UP ? 4 : 0);
    constexpr int kNK = kSpatial + (TEMP ? 25 : 0);
    __shared__ float sN[3][kHY][kHX];
    __shared__ float sW[TEMP ? 3 : 1][TEMP ? kHY : 1][TEMP ? kHX : 1];

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    const int bx0 = blockIdx.x * kTX, by0 = blockIdx.y * kTY;
    const int x = bx0 + tx, y = by0 + ty;
    const bool inside = x < Wl && y < Hl;
    const int xc = x < Wl ? x : Wl - 1;
    const int yc = y < Hl ? y : Hl - 1;
    const long long Nl = static_cast<long long>(Wl) * Hl;
    const long long pix = static_cast<long long>(yc) * Wl + xc;

    // logits first: the longest-latency, largest stream
    float lg[kNK];
#pragma unroll
    for (int k = 0; k < kSpatial; ++k) lg[k] = __ldcs(logits + k * Nl + pix);
    bool use_t = false;
    if (TEMP) {
        use_t = !(mask && mask[pix]);
        if (use_t) {
#pragma unroll
            for (int k = 0; k < 25; ++k) lg[kSpatial + k] = __ldcs(logits + (29 + k) * Nl + pix);
        } else {
#pragma unroll
            for (int k = 0; k < 25; ++k) lg[kSpatial + k] = 0.0f;
        }
    }

    // stage the noisy tile (+ halo) and, at full resolution, the warped
    // previous frame on the same halo, clamped to the edge
    for (int idx = tid; idx < kHX * kHY; idx += kTX * kTY) {
        const int hx = idx % kHX, hy = idx / kHX;
        const int gx = clampi(bx0 + hx - kHalo, 0, Wl - 1);
        const int gy = clampi(by0 + hy - kHalo, 0, Hl - 1);
        const long long g = static_cast<long long>(gy) * Wl + gx;
        sN[0][hy][hx] = __ldg(noisy + g);
        sN[1][hy][hx] = __ldg(noisy + Nl + g);
        sN[2][hy][hx] = __ldg(noisy + 2 * Nl + g);
        if (TEMP) {
            sW[0][hy][hx] = __ldg(warped + g);
            sW[1][hy][hx] = __ldg(warped + Nl + g);
            sW[2][hy][hx] = __ldg(warped + 2 * Nl + g);
        }
    }
    __syncthreads();

    // joint softmax over the kernels present at this pixel
    float m = lg[0];
#pragma unroll
    for (int k = 1; k < kSpatial; ++k) m = fmaxf(m, lg[k]);
    if (TEMP && use_t) {
#pragma unroll
        for (int k = kSpatial; k < kNK; ++k) m = fmaxf(m, lg[k]);
    }
    const float mL = m * kLog2e;
    float wsum = 0.0f, a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
    // G(L^l, kappa_d), Eq. app-gather
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float e = exp2f(fmaf(lg[j * 5 + i], kLog2e, -mL));
            wsum += e;
            a0 = fmaf(e, sN[0][ty + j][tx + i], a0);
            a1 = fmaf(e, sN[1][ty + j][tx + i], a1);
            a2 = fmaf(e, sN[2][ty + j][tx + i], a2);
        }
    // U(L-hat^{l+1}, kappa_u), Eq. app-upsample: taps at floor((x+i)/2)
    if (UP) {
        const int Wc = Wl >> 1, Hc = Hl >> 1;
        const long long Nc = static_cast<long long>(Wc) * Hc;
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int cx = min((xc + i) >> 1, Wc - 1), cy = min((yc + j) >> 1, Hc - 1);
                const long long q = static_cast<long long>(cy) * Wc + cx;
                const float e = exp2f(fmaf(lg[25 + 2 * j + i], kLog2e, -mL));
                wsum += e;
                a0 = fmaf(e, __ldg(coarse + q), a0);
                a1 = fmaf(e, __ldg(coarse + Nc + q), a1);
                a2 = fmaf(e, __ldg(coarse + 2 * Nc + q), a2);
            }
    }
    // G(W_t L_{t-1}, kappa_t), Eq. app-recon-full
    if (TEMP && use_t) {
#pragma unroll
        for (int j = 0; j < 5; ++j)
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                const float e = exp2f(fmaf(lg[kSpatial + j * 5 + i], kLog2e, -mL));
                wsum += e;
                a0 = fmaf(e, sW[0][ty + j][tx + i], a0);
                a1 = fmaf(e, sW[1][ty + j][tx + i], a1);
                a2 = fmaf(e, sW[2][ty + j][tx + i], a2);
            }
    }
    const float inv = rcp_approx(wsum);
    const float o0 = a0 * inv, o1 = a1 * inv, o2 = a2 * inv;
    if (!inside) return;
    const long long op = static_cast<long long>(y) * Wl + x;
    __stcs(out + op, o0);
    __stcs(out + Nl + op, o1);
    __stcs(out + 2 * Nl + op, o2);
    if (TONE) {
        float r, g, b;
        tone_map(o0, o1, o2, tm, r, g, b);
        __stcs(out_ldr + op, r);
        __stcs(out_ldr + Nl + op, g);
        __stcs(out_ldr + 2 * Nl + op, b);
    }
}

template <bool UP, bool TEMP>
void launch_level(bool tone, dim3 grid, dim3 block, cudaStream_t st, const float *noisy,
                  const float *logits, const float *coarse, const float *warped,
                  const uint8_t *mask, int Wl, int Hl, float *out, float *out_ldr,
                  const ToneArgs &tm) {
    if (tone)
        recon_kernel<UP, TEMP, true><<<grid, block, 0, st>>>(noisy, logits, coarse, warped, mask,
                                                             Wl, Hl, out, out_ldr, tm);
    else
        recon_kernel<UP, TEMP, false><<<grid, block, 0, st>>>(noisy, logits, coarse, warped, mask,
                                                              Wl, Hl, out, out_ldr, tm);
}

// Tone map of a whole HDR image (Sec. 5), for reference images and the
// recurrent network input.
__global__ void tonemap_image_kernel(const float *__restrict__ hdr, int64_t n,
                                     float *__restrict__ ldr, ToneArgs tm) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        float r, g, b;
        tone_map(hdr[i], hdr[n + i], hdr[2 * n + i], tm, r, g, b);
        ldr[i] = r;
        ldr[n + i] = g;
        ldr[2 * n + i] = b;
    }
}

size_t align256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

}  // namespace

// Tone-map arguments of a call (defaults when tm is NULL) and their check;
// also used by the two-stage pipeline's remodulation.
ToneArgs tone_args(const spp_tonemap *tm) {
    ToneArgs t{1.0f, 1.0f, 0.0f, 0.5f, 0.5f, 2.0f, 2.0f};
    if (tm) {
        t.alpha = tm->alpha;
        t.beta = tm->beta;
        t.k = tm->exposure;
        t.s = tm->shadow;
        t.h = tm->highlight;
    }
    t.inv_s = 1.0f / t.s;
    t.inv_h = 1.0f / t.h;
    return t;
}

bool tone_ok(const ToneArgs &t) {
    return t.s > 0.0f && t.s < 1.0f && t.h > 0.0f && t.h < 1.0f && t.alpha == t.alpha &&
           t.beta == t.beta && t.k == t.k;
}

}  // namespace spp

extern "C" {

int spp_tonemap_image(const float *hdr, int W, int H, const spp_tonemap *tm, float *ldr,
                      cudaStream_t stream) {
    using namespace spp;
    if (W < 0 || H < 0 || !hdr || !ldr) return SPP_ERR_ARG;
    if (!aligned16(hdr) || !aligned16(ldr)) return SPP_ERR_ALIGN;
    const ToneArgs t = tone_args(tm);
    if (!tone_ok(t)) return SPP_ERR_ARG;
    const int64_t n = static_cast<int64_t>(W) * H;
    if (n == 0) return SPP_OK;
    const int grid = static_cast<int>(std::min<int64_t>((n + 255) / 256, 8 * sm_count()));
    tonemap_image_kernel<<<grid, 256, 0, stream>>>(hdr, n, ldr, t);
    count_launch();
    return launch_status();
}

int spp_warp_previous(const float *prev_hdr, const float *mv, int W, int H, float *warped,
                      cudaStream_t stream) {
    using namespace spp;
    if (W < 0 || H < 0 || !prev_hdr || !mv || !warped) return SPP_ERR_ARG;
    if (!aligned16(prev_hdr) || !aligned16(mv) || !aligned16(warped)) return SPP_ERR_ALIGN;
    if (static_cast<long long>(W) * H == 0) return SPP_OK;
    launch_warp_prev(prev_hdr, mv, W, H, warped, stream);
    count_launch();
    return launch_status();
}

int spp_reconstruct_level(const float *noisy, const float *logits, int C, const float *coarse,
                          const float *warped_prev, const uint8_t *mask, int Wl, int Hl,
                          const spp_tonemap *tm, float *out, float *out_ldr, int32_t *status,
                          cudaStream_t stream) {
    using namespace spp;
    if (Wl < 0 || Hl < 0 || !noisy || !logits || !out) return SPP_ERR_ARG;
    if (warped_prev && !coarse) return SPP_ERR_ARG;
    const int need = 25 + (coarse ? 4 : 0);
    if (C < need || (warped_prev && C < 54)) return SPP_ERR_ARG;
    if (coarse && ((Wl & 1) || (Hl & 1))) return SPP_ERR_SHAPE;
    if (!aligned16(noisy) || !aligned16(logits) || !aligned16(out) ||
        (coarse && !aligned16(coarse)) || (warped_prev && !aligned16(warped_prev)) ||
        (mask && !aligned16(mask)) || (out_ldr && !aligned16(out_ldr)) ||
        (status && !aligned16(status)))
        return SPP_ERR_ALIGN;
    const ToneArgs ta = tone_args(tm);
    if (out_ldr && !tone_ok(ta)) return SPP_ERR_ARG;
    if (static_cast<long long>(Wl) * Hl == 0) return SPP_OK;
    const int C_used = warped_prev ? 54 : (coarse ? 29 : 25);
    int rc = SPP_OK;
    if (launch_recon_tma(noisy, logits, C, C_used, coarse, warped_prev, mask, Wl, Hl, out, out_ldr,
                         ta, status, stream, &rc))
        return rc;
    dim3 block(kTX, kTY);
    dim3 grid((Wl + kTX - 1) / kTX, (Hl + kTY - 1) / kTY);
    const bool tone = out_ldr != nullptr;
    if (!coarse)
        launch_level<false, false>(tone, grid, block, stream, noisy, logits, coarse, warped_prev,
                                   mask, Wl, Hl, out, out_ldr, ta);
    else if (!warped_prev)
        launch_level<true, false>(tone, grid, block, stream, noisy, logits, coarse, warped_prev,
                                  mask, Wl, Hl, out, out_ldr, ta);
    else
        launch_level<true, true>(tone, grid, block, stream, noisy, logits, coarse, warped_prev,
                                 mask, Wl, Hl, out, out_ldr, ta);
    count_launch();
    return launch_status();
}

size_t spp_reconstruct_workspace_bytes(int W, int H, int L) {
    if (W < 0 || H < 0 || L < 2 || L > 5) return 0;
    size_t total = spp::align256(3 * sizeof(float) * static_cast<size_t>(W) *
                                 static_cast<size_t>(H));  // W_t L_{t-1}
    for (int l = 1; l < L; ++l)
        total += spp::align256(3 * sizeof(float) * static_cast<size_t>(W >> l) *
                               static_cast<size_t>(H >> l));
    return total;
}

int spp_reconstruct_frame(const float *const *layers, const float *const *logits, int C0,
                          const float *prev_hdr, const float *mv, const uint8_t *mask, int W,
                          int H, int L, const spp_tonemap *tm, float *out_hdr, float *out_ldr,
                          void *ws, size_t ws_bytes, int32_t *status, cudaStream_t stream) {
    using namespace spp;
    if (!layers || !logits || !out_hdr || W < 0 || H < 0) return SPP_ERR_ARG;
    if (L < 2 || L > 5) return SPP_ERR_SHAPE;
    if ((W % (1 << (L - 1))) != 0 || (H % (1 << (L - 1))) != 0) return SPP_ERR_SHAPE;
    if (C0 != 29 && C0 != 54) return SPP_ERR_ARG;
    if (prev_hdr && C0 != 54) return SPP_ERR_ARG;
    for (int l = 0; l < L; ++l)
        if (!layers[l] || !logits[l]) return SPP_ERR_ARG;
    const size_t need = spp_reconstruct_workspace_bytes(W, H, L);
    if (ws_bytes < need || (need && !ws)) return SPP_ERR_WORKSPACE;
    if (ws && !aligned16(ws)) return SPP_ERR_ALIGN;
    float *hat[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    float *warped = static_cast<float *>(ws);
    size_t off = align256(3 * sizeof(float) * static_cast<size_t>(W) * static_cast<size_t>(H));
    for (int l = 1; l < L; ++l) {
        hat[l] = reinterpret_cast<float *>(static_cast<char *>(ws) + off);
        off += align256(3 * sizeof(float) * static_cast<size_t>(W >> l) * static_cast<size_t>(H >> l));
    }
    for (int l = L - 1; l >= 1; --l) {
        const int C = (l == L - 1) ? 25 : 29;
        const int rc = spp_reconstruct_level(layers[l], logits[l], C, l == L - 1 ? nullptr : hat[l + 1],
                                             nullptr, nullptr, W >> l, H >> l, nullptr, hat[l],
                                             nullptr, status, stream);
        if (rc != SPP_OK) return rc;
    }
    if (prev_hdr) {
        if (!mv) return SPP_ERR_ARG;
        const int rc = spp_warp_previous(prev_hdr, mv, W, H, warped, stream);
        if (rc != SPP_OK) return rc;
    }
    return spp_reconstruct_level(layers[0], logits[0], C0, hat[1], prev_hdr ? warped : nullptr,
                                 prev_hdr ? mask : nullptr, W, H, tm, out_hdr, out_ldr, status,
                                 stream);
}

}  // extern "C"
