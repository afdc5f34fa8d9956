// a6-a9: gather-pyramid reconstruction (Appendix A of arXiv 2602.08642) with
// the temporal term over the bilinearly reprojected previous output and the
// filmic tone map + sRGB epilogue (Sec. 5).
//
// One kernel per pyramid level.  A block owns a 32 x 8 pixel tile: it stages
// the noisy level's tile plus a 2-pixel halo in shared memory and, at full
// resolution, the warped previous frame W_t L_{t-1} on the same halo (each
// halo pixel warped with its own motion vector), so that the 5 x 5 gathers
// read shared memory.  The per-pixel logits (the dominant HBM stream: 54
// planes at full resolution) are read once, coalesced along x, and the joint
// softmax is evaluated in registers.
#include "spp_internal.cuh"

namespace spp {
namespace {

constexpr int kTX = 32;
constexpr int kTY = 8;
constexpr int kHalo = 2;
constexpr int kHX = kTX + 2 * kHalo;
constexpr int kHY = kTY + 2 * kHalo;
constexpr float kLog2e = 1.4426950408889634f;

struct ToneArgs {
    float alpha, beta, k, s, h;
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// tau of Sec. 5: exponential toe below s-1, linear middle, exponential shoulder
// above 1-h.
__device__ __forceinline__ float tau_curve(float x, float s, float h) {
    if (x < s - 1.0f) return 0.5f * s * __expf((x + 1.0f - s) / s);
    if (x < 1.0f - h) return 0.5f * (1.0f + x);
    return 1.0f - 0.5f * h * __expf(-(x + h - 1.0f) / h);
}

// IEC 61966-2-1 sRGB encoding.
__device__ __forceinline__ float srgb(float v) {
    return v <= 0.0031308f ? 12.92f * v : 1.055f * __powf(v, 1.0f / 2.4f) - 0.055f;
}

template <bool UP, bool TEMP, bool TONE>
__global__ void __launch_bounds__(kTX *kTY, 2)
recon_kernel(const float *__restrict__ noisy, const float *__restrict__ logits,
             const float *__restrict__ coarse, const float *__restrict__ prev,
             const float *__restrict__ mv, const uint8_t *__restrict__ mask, int Wl, int Hl,
             float *__restrict__ out, float *__restrict__ out_ldr, ToneArgs tm) {
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
    // previous frame on the same halo
    for (int idx = tid; idx < kHX * kHY; idx += kTX * kTY) {
        const int hx = idx % kHX, hy = idx / kHX;
        const int gx = clampi(bx0 + hx - kHalo, 0, Wl - 1);
        const int gy = clampi(by0 + hy - kHalo, 0, Hl - 1);
        const long long g = static_cast<long long>(gy) * Wl + gx;
        sN[0][hy][hx] = __ldg(noisy + g);
        sN[1][hy][hx] = __ldg(noisy + Nl + g);
        sN[2][hy][hx] = __ldg(noisy + 2 * Nl + g);
        if (TEMP) {
            // W_t: bilinear at (gx + mv_x, gy + mv_y), pixel centres at
            // integers, position clamped to the frame.  The fraction is taken
            // from the motion vector itself so that it is exact.
            const float mx = __ldg(mv + g), my = __ldg(mv + Nl + g);
            float ix = fminf(fmaxf(floorf(mx), -1048576.0f), 1048576.0f);
            float iy = fminf(fmaxf(floorf(my), -1048576.0f), 1048576.0f);
            float fx = mx - floorf(mx), fy = my - floorf(my);
            int X0 = gx + static_cast<int>(ix), Y0 = gy + static_cast<int>(iy);
            if (X0 < 0) { X0 = 0; fx = 0.0f; } else if (X0 >= Wl - 1) { X0 = Wl - 1; fx = 0.0f; }
            if (Y0 < 0) { Y0 = 0; fy = 0.0f; } else if (Y0 >= Hl - 1) { Y0 = Hl - 1; fy = 0.0f; }
            const int X1 = X0 + 1 < Wl ? X0 + 1 : Wl - 1;
            const int Y1 = Y0 + 1 < Hl ? Y0 + 1 : Hl - 1;
            const long long r0 = static_cast<long long>(Y0) * Wl, r1 = static_cast<long long>(Y1) * Wl;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float *P = prev + c * Nl;
                const float p00 = __ldg(P + r0 + X0), p10 = __ldg(P + r0 + X1);
                const float p01 = __ldg(P + r1 + X0), p11 = __ldg(P + r1 + X1);
                sW[c][hy][hx] = (1.0f - fy) * ((1.0f - fx) * p00 + fx * p10) +
                                fy * ((1.0f - fx) * p01 + fx * p11);
            }
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
    const float inv = __frcp_rn(wsum);
    const float o0 = a0 * inv, o1 = a1 * inv, o2 = a2 * inv;
    if (!inside) return;
    const long long op = static_cast<long long>(y) * Wl + x;
    __stcs(out + op, o0);
    __stcs(out + Nl + op, o1);
    __stcs(out + 2 * Nl + op, o2);
    if (TONE) {
        // Sec. 5: x_c = alpha (mean + beta (ln L_c - mean) + k), then tau, sRGB
        const float l0 = __logf(fmaxf(o0, 0x1p-24f));
        const float l1 = __logf(fmaxf(o1, 0x1p-24f));
        const float l2 = __logf(fmaxf(o2, 0x1p-24f));
        const float mean = (l0 + l1 + l2) * (1.0f / 3.0f);
        const float x0v = tm.alpha * (mean + tm.beta * (l0 - mean) + tm.k);
        const float x1v = tm.alpha * (mean + tm.beta * (l1 - mean) + tm.k);
        const float x2v = tm.alpha * (mean + tm.beta * (l2 - mean) + tm.k);
        __stcs(out_ldr + op, srgb(tau_curve(x0v, tm.s, tm.h)));
        __stcs(out_ldr + Nl + op, srgb(tau_curve(x1v, tm.s, tm.h)));
        __stcs(out_ldr + 2 * Nl + op, srgb(tau_curve(x2v, tm.s, tm.h)));
    }
}

template <bool UP, bool TEMP>
void launch_level(bool tone, dim3 grid, dim3 block, cudaStream_t st, const float *noisy,
                  const float *logits, const float *coarse, const float *prev, const float *mv,
                  const uint8_t *mask, int Wl, int Hl, float *out, float *out_ldr,
                  const ToneArgs &tm) {
    if (tone)
        recon_kernel<UP, TEMP, true><<<grid, block, 0, st>>>(noisy, logits, coarse, prev, mv, mask,
                                                             Wl, Hl, out, out_ldr, tm);
    else
        recon_kernel<UP, TEMP, false><<<grid, block, 0, st>>>(noisy, logits, coarse, prev, mv,
                                                              mask, Wl, Hl, out, out_ldr, tm);
}

ToneArgs tone_args(const spp_tonemap *tm) {
    ToneArgs t{1.0f, 1.0f, 0.0f, 0.5f, 0.5f};
    if (tm) {
        t.alpha = tm->alpha;
        t.beta = tm->beta;
        t.k = tm->exposure;
        t.s = tm->shadow;
        t.h = tm->highlight;
    }
    return t;
}

bool tone_ok(const ToneArgs &t) {
    return t.s > 0.0f && t.s < 1.0f && t.h > 0.0f && t.h < 1.0f && t.alpha == t.alpha &&
           t.beta == t.beta && t.k == t.k;
}

size_t align256(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

}  // namespace
}  // namespace spp

extern "C" {

int spp_reconstruct_level(const float *noisy, const float *logits, int C, const float *coarse,
                          const float *prev_hdr, const float *mv, const uint8_t *mask, int Wl,
                          int Hl, const spp_tonemap *tm, float *out, float *out_ldr,
                          cudaStream_t stream) {
    using namespace spp;
    if (Wl < 0 || Hl < 0 || !noisy || !logits || !out) return SPP_ERR_ARG;
    if (prev_hdr && (!coarse || !mv)) return SPP_ERR_ARG;
    const int need = 25 + (coarse ? 4 : 0);
    if (C < need || (prev_hdr && C < 54)) return SPP_ERR_ARG;
    if (coarse && ((Wl & 1) || (Hl & 1))) return SPP_ERR_SHAPE;
    if (!aligned16(noisy) || !aligned16(logits) || !aligned16(out) ||
        (coarse && !aligned16(coarse)) || (prev_hdr && !aligned16(prev_hdr)) ||
        (mv && !aligned16(mv)) || (mask && !aligned16(mask)) || (out_ldr && !aligned16(out_ldr)))
        return SPP_ERR_ALIGN;
    const ToneArgs ta = tone_args(tm);
    if (out_ldr && !tone_ok(ta)) return SPP_ERR_ARG;
    if (static_cast<long long>(Wl) * Hl == 0) return SPP_OK;
    dim3 block(kTX, kTY);
    dim3 grid((Wl + kTX - 1) / kTX, (Hl + kTY - 1) / kTY);
    const bool tone = out_ldr != nullptr;
    if (!coarse)
        launch_level<false, false>(tone, grid, block, stream, noisy, logits, coarse, prev_hdr, mv,
                                   mask, Wl, Hl, out, out_ldr, ta);
    else if (!prev_hdr)
        launch_level<true, false>(tone, grid, block, stream, noisy, logits, coarse, prev_hdr, mv,
                                  mask, Wl, Hl, out, out_ldr, ta);
    else
        launch_level<true, true>(tone, grid, block, stream, noisy, logits, coarse, prev_hdr, mv,
                                 mask, Wl, Hl, out, out_ldr, ta);
    count_launch();
    return launch_status();
}

size_t spp_reconstruct_workspace_bytes(int W, int H, int L) {
    if (W < 0 || H < 0 || L < 2 || L > 5) return 0;
    size_t total = 0;
    for (int l = 1; l < L; ++l)
        total += spp::align256(3 * sizeof(float) * static_cast<size_t>(W >> l) *
                               static_cast<size_t>(H >> l));
    return total;
}

int spp_reconstruct_frame(const float *const *layers, const float *const *logits, int C0,
                          const float *prev_hdr, const float *mv, const uint8_t *mask, int W,
                          int H, int L, const spp_tonemap *tm, float *out_hdr, float *out_ldr,
                          void *ws, size_t ws_bytes, cudaStream_t stream) {
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
    size_t off = 0;
    for (int l = 1; l < L; ++l) {
        hat[l] = reinterpret_cast<float *>(static_cast<char *>(ws) + off);
        off += align256(3 * sizeof(float) * static_cast<size_t>(W >> l) * static_cast<size_t>(H >> l));
    }
    for (int l = L - 1; l >= 1; --l) {
        const int C = (l == L - 1) ? 25 : 29;
        const int rc = spp_reconstruct_level(layers[l], logits[l], C, l == L - 1 ? nullptr : hat[l + 1],
                                             nullptr, nullptr, nullptr, W >> l, H >> l, nullptr,
                                             hat[l], nullptr, stream);
        if (rc != SPP_OK) return rc;
    }
    return spp_reconstruct_level(layers[0], logits[0], C0, hat[1], prev_hdr, prev_hdr ? mv : nullptr,
                                 prev_hdr ? mask : nullptr, W, H, tm, out_hdr, out_ldr, stream);
}

}  // extern "C"
