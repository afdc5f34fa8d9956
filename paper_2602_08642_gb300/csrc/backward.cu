// a11: backward pass of the sampling + reconstruction path (arXiv 2602.08642):
// the joint-softmax gather pyramid (App. A), the reprojection W_t, the tone
// map (Sec. 5), the L1 loss in sRGB (Eq. loss_spatial with m = 1), the
// average-pool pyramid, the density-normalised splat with the relaxed ramp
// (Eq. stoch_rnoisy, Eq. relaxed_holdout) and the spatial softmax of the
// sampler output (Sec. 3).
//
// The reconstruction backward recomputes each pixel's softmax weights from
// its logits instead of storing the K x K tap products, and takes the
// transpose of the gathers in gather form (each source pixel sums the
// contributions of the pixels that read it, in a fixed order): its result
// is the same from run to run.  The bilinear warp's backward scatters with
// atomics (a source pixel's readers are not bounded for arbitrary motion),
// and so may differ in its last bits from run to run.
#include "recon_common.cuh"
#include "render_common.cuh"

namespace spp {
namespace {

constexpr int kBX = 32, kBY = 8, kBH = 2;
constexpr int kRX = kBX + 2 * kBH, kRY = kBY + 2 * kBH;  // consumer region 36 x 12
constexpr int kRN = kRX * kRY;                           // 432 consumers
constexpr int kHalo = kRN - kBX * kBY;                   // 176 of them outside the tile
constexpr int kFX = kBX / 2 + 1, kFY = kBY / 2 + 1;      // coarse cells the tile's taps read

// Shared memory of the backward of one 32 x 8 tile: per consumer pixel of
// the tile and its 2-pixel halo the normalised weights of its kernels and
// dLoss/d out; the tap values the tile's own pixels read.
template <bool UP, bool TEMP>
struct BwdSmem {
    float wd[25][kRN];
    float wu[UP ? 4 : 1][UP ? kRN : 1];
    float wt[TEMP ? 25 : 1][TEMP ? kRN : 1];
    float g[3][kRN];
    float nz[3][kRN];
    float wp[TEMP ? 3 : 1][TEMP ? kRN : 1];
    float cv[UP ? 3 : 1][UP ? kFY * kFX : 1];
};

// Taps i in [lo, hi] of a consumer at q whose clamped source, clamp(q + i -
// 2) to [0, n - 1], is p (the transpose of clamp-to-edge along one axis);
// lo > hi when there is none.
__device__ __forceinline__ void tap_range(int q, int p, int n, int &lo, int &hi) {
    if (n == 1) {
        lo = 0;
        hi = 4;
    } else if (p == 0) {
        lo = 0;
        hi = min(2 - q, 4);
    } else if (p == n - 1) {
        lo = max(n + 1 - q, 0);
        hi = 4;
    } else {
        lo = hi = p - q + 2;
        if (lo < 0 || lo > 4) hi = lo - 1;
    }
}

// Backward of one reconstruction level in gather form: every output
// gradient element has exactly one writer, which adds its consumers'
// contributions in a fixed order, so the result does not depend on
// scheduling.  A block owns a 32 x 8 tile: it computes the softmax weights
// of the tile's pixels and of the 2-pixel halo around it (the consumers of
// the tile's sources), dLoss/d logits of the tile's pixels, then for each
// source pixel of the tile (and for each coarse cell under it) the sum of
// w_k g over the consumers and taps that read it.
template <bool UP, bool TEMP>
__global__ void __launch_bounds__(kBX *kBY)
recon_backward_kernel(const float *__restrict__ noisy, const float *__restrict__ logits, int C,
                      const float *__restrict__ coarse, const float *__restrict__ warped,
                      const uint8_t *__restrict__ mask, int Wl, int Hl,
                      const float *__restrict__ g, float *__restrict__ grad_logits,
                      float *__restrict__ grad_noisy, float *__restrict__ grad_coarse,
                      float *__restrict__ grad_warped) {
    constexpr int kSpatial = 25 + (UP ? 4 : 0);
    constexpr int kNK = kSpatial + (TEMP ? 25 : 0);
    extern __shared__ __align__(16) unsigned char bwd_smem_raw[];
    BwdSmem<UP, TEMP> &sm = *reinterpret_cast<BwdSmem<UP, TEMP> *>(bwd_smem_raw);

    const int tid = threadIdx.y * kBX + threadIdx.x;
    const int bx0 = blockIdx.x * kBX, by0 = blockIdx.y * kBY;
    const long long Nl = static_cast<long long>(Wl) * Hl;
    const int Wc = Wl >> 1, Hc = Hl >> 1;
    const long long Nc = static_cast<long long>(Wc) * Hc;
    const int cbx = bx0 >> 1, cby = by0 >> 1;  // first coarse cell under the tile

    // tap values of the region (clamp-to-edge)
    for (int idx = tid; idx < kRN; idx += kBX * kBY) {
        const int rx = idx % kRX, ry = idx / kRX;
        const int gx = clampi(bx0 + rx - kBH, 0, Wl - 1), gy = clampi(by0 + ry - kBH, 0, Hl - 1);
        const long long q = static_cast<long long>(gy) * Wl + gx;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sm.nz[c][idx] = __ldg(noisy + c * Nl + q);
            if (TEMP) sm.wp[c][idx] = __ldg(warped + c * Nl + q);
        }
    }
    if (UP)
        for (int idx = tid; idx < kFX * kFY; idx += kBX * kBY) {
            const int cx = min(cbx + idx % kFX, Wc - 1), cy = min(cby + idx / kFX, Hc - 1);
            const long long q = static_cast<long long>(cy) * Wc + cx;
#pragma unroll
            for (int c = 0; c < 3; ++c) sm.cv[c][idx] = __ldg(coarse + c * Nc + q);
        }

    // the normalised weights and dLoss/d out of consumer (qx, qy) into its
    // region cell; w receives them for the caller
    auto consumer = [&](int qx, int qy, int cell, float (&w)[kNK], float (&gq)[3], bool &use_t) {
        const bool in = qx >= 0 && qx < Wl && qy >= 0 && qy < Hl;
        use_t = false;
        if (!in) {  // not a pixel: reads nothing, contributes nothing
#pragma unroll
            for (int k = 0; k < kNK; ++k) w[k] = 0.0f;
            gq[0] = gq[1] = gq[2] = 0.0f;
        } else {
            const long long pix = static_cast<long long>(qy) * Wl + qx;
            use_t = TEMP && !(mask && mask[pix]);
#pragma unroll
            for (int k = 0; k < kSpatial; ++k) w[k] = __ldg(logits + k * Nl + pix);
            if (TEMP) {
#pragma unroll
                for (int k = 0; k < 25; ++k)
                    w[kSpatial + k] = use_t ? __ldg(logits + (29 + k) * Nl + pix) : 0.0f;
            }
            float m = w[0];
#pragma unroll
            for (int k = 1; k < kSpatial; ++k) m = fmaxf(m, w[k]);
            if (use_t) {
#pragma unroll
                for (int k = kSpatial; k < kNK; ++k) m = fmaxf(m, w[k]);
            }
            float wsum = 0.0f;
#pragma unroll
            for (int k = 0; k < kNK; ++k) {
                const bool on = k < kSpatial || use_t;
                w[k] = on ? __expf(w[k] - m) : 0.0f;
                wsum += w[k];
            }
            const float inv = 1.0f / wsum;
#pragma unroll
            for (int k = 0; k < kNK; ++k) w[k] *= inv;
#pragma unroll
            for (int c = 0; c < 3; ++c) gq[c] = __ldg(g + c * Nl + pix);
        }
#pragma unroll
        for (int k = 0; k < 25; ++k) sm.wd[k][cell] = w[k];
        if (UP) {
#pragma unroll
            for (int k = 0; k < 4; ++k) sm.wu[k][cell] = w[25 + k];
        }
        if (TEMP) {
#pragma unroll
            for (int k = 0; k < 25; ++k) sm.wt[k][cell] = w[kSpatial + k];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) sm.g[c][cell] = gq[c];
    };
    __syncthreads();

    // the tile's own pixel: its weights, then dLoss/d logits
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int px = bx0 + tx, py = by0 + ty;
    const bool inside = px < Wl && py < Hl;
    {
        float w[kNK], gq[3];
        bool use_t;
        const int cell = (ty + kBH) * kRX + tx + kBH;
        consumer(px, py, cell, w, gq, use_t);
        if (inside) {
            const long long pix = static_cast<long long>(py) * Wl + px;
            float q[kNK];
#pragma unroll
            for (int j = 0; j < 5; ++j)
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    const int o = (ty + j) * kRX + tx + i;
                    q[j * 5 + i] =
                        gq[0] * sm.nz[0][o] + gq[1] * sm.nz[1][o] + gq[2] * sm.nz[2][o];
                    if (TEMP)
                        q[kSpatial + j * 5 + i] =
                            gq[0] * sm.wp[0][o] + gq[1] * sm.wp[1][o] + gq[2] * sm.wp[2][o];
                }
            if (UP) {
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int cx = min((px + i) >> 1, Wc - 1) - cbx;
                        const int cy = min((py + j) >> 1, Hc - 1) - cby;
                        const int o = cy * kFX + cx;
                        q[25 + 2 * j + i] =
                            gq[0] * sm.cv[0][o] + gq[1] * sm.cv[1][o] + gq[2] * sm.cv[2][o];
                    }
            }
            float qbar = 0.0f;
#pragma unroll
            for (int k = 0; k < kNK; ++k) qbar = fmaf(w[k], q[k], qbar);
            // dLoss/dz_k = w_k (q_k - qbar); channels without a kernel get 0
#pragma unroll
            for (int k = 0; k < kSpatial; ++k) grad_logits[k * Nl + pix] = w[k] * (q[k] - qbar);
            if (TEMP) {
#pragma unroll
                for (int k = 0; k < 25; ++k)
                    grad_logits[(29 + k) * Nl + pix] =
                        use_t ? w[kSpatial + k] * (q[kSpatial + k] - qbar) : 0.0f;
            }
            for (int k = TEMP ? 54 : kSpatial; k < C; ++k) grad_logits[k * Nl + pix] = 0.0f;
        }
    }
    // the halo's consumers (rows 0-1 and 10-11, then columns 0-1 and 34-35)
    if (tid < kHalo) {
        int rx, ry;
        if (tid < 2 * kRX) {
            rx = tid % kRX;
            ry = tid / kRX;
        } else if (tid < 4 * kRX) {
            rx = (tid - 2 * kRX) % kRX;
            ry = kRY - 2 + (tid - 2 * kRX) / kRX;
        } else {
            const int h = tid - 4 * kRX;
            ry = kBH + h / 4;
            rx = (h % 4) < 2 ? (h % 4) : kBX + (h % 4);
        }
        float w[kNK], gq[3];
        bool use_t;
        consumer(bx0 + rx - kBH, by0 + ry - kBH, ry * kRX + rx, w, gq, use_t);
    }
    __syncthreads();

    // sources of the tile: the sum of w_k g over the taps that read them
    if (inside && (grad_noisy || (TEMP && grad_warped))) {
        float an[3] = {0.0f, 0.0f, 0.0f}, aw[3] = {0.0f, 0.0f, 0.0f};
        // CTA-uniform: every source of the tile is 2 or more pixels from the
        // border, so each consumer reads it through exactly one tap
        const bool inner = bx0 >= 2 && bx0 + kBX + 2 <= Wl && by0 >= 2 && by0 + kBY + 2 <= Hl;
        if (inner) {
#pragma unroll
            for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
                for (int dx = -2; dx <= 2; ++dx) {
                    const int cell = (ty + kBH + dy) * kRX + tx + kBH + dx;
                    const int k = (2 - dy) * 5 + (2 - dx);
                    const float wk = sm.wd[k][cell];
#pragma unroll
                    for (int c = 0; c < 3; ++c) an[c] = fmaf(wk, sm.g[c][cell], an[c]);
                    if (TEMP) {
                        const float wt = sm.wt[k][cell];
#pragma unroll
                        for (int c = 0; c < 3; ++c) aw[c] = fmaf(wt, sm.g[c][cell], aw[c]);
                    }
                }
        } else {
            for (int dy = -2; dy <= 2; ++dy) {
                const int qy = py + dy;
                if (qy < 0 || qy >= Hl) continue;
                int jlo, jhi;
                tap_range(qy, py, Hl, jlo, jhi);
                for (int dx = -2; dx <= 2; ++dx) {
                    const int qx = px + dx;
                    if (qx < 0 || qx >= Wl) continue;
                    int ilo, ihi;
                    tap_range(qx, px, Wl, ilo, ihi);
                    const int cell = (ty + kBH + dy) * kRX + tx + kBH + dx;
                    for (int j = jlo; j <= jhi; ++j)
                        for (int i = ilo; i <= ihi; ++i) {
                            const float wk = sm.wd[j * 5 + i][cell];
#pragma unroll
                            for (int c = 0; c < 3; ++c) an[c] = fmaf(wk, sm.g[c][cell], an[c]);
                            if (TEMP) {
                                const float wt = sm.wt[j * 5 + i][cell];
#pragma unroll
                                for (int c = 0; c < 3; ++c)
                                    aw[c] = fmaf(wt, sm.g[c][cell], aw[c]);
                            }
                        }
                }
            }
        }
        const long long pix = static_cast<long long>(py) * Wl + px;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (grad_noisy) grad_noisy[c * Nl + pix] += an[c];
            if (TEMP && grad_warped) grad_warped[c * Nl + pix] += aw[c];
        }
    }
    // coarse cells under the tile: the upsampling taps of the full-resolution
    // pixels 2c - 1 .. 2c + 1 that read them
    if (UP && grad_coarse && tid < (kBX / 2) * (kBY / 2)) {
        const int cx = cbx + tid % (kBX / 2), cy = cby + tid / (kBX / 2);
        if (cx < Wc && cy < Hc) {
            float ac[3] = {0.0f, 0.0f, 0.0f};
            for (int qy = 2 * cy - 1; qy <= 2 * cy + 1; ++qy) {
                if (qy < 0 || qy >= Hl) continue;
                for (int qx = 2 * cx - 1; qx <= 2 * cx + 1; ++qx) {
                    if (qx < 0 || qx >= Wl) continue;
                    const int cell = (qy - by0 + kBH) * kRX + qx - bx0 + kBH;
#pragma unroll
                    for (int j = 0; j < 2; ++j)
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            if (min((qx + i) >> 1, Wc - 1) != cx || min((qy + j) >> 1, Hc - 1) != cy)
                                continue;
                            const float wk = sm.wu[2 * j + i][cell];
#pragma unroll
                            for (int c = 0; c < 3; ++c) ac[c] = fmaf(wk, sm.g[c][cell], ac[c]);
                        }
                }
            }
            const long long q = static_cast<long long>(cy) * Wc + cx;
#pragma unroll
            for (int c = 0; c < 3; ++c) grad_coarse[c * Nc + q] += ac[c];
        }
    }
}

// W_t backward: each pixel's bilinear weights scatter its gradient to the
// four previous-frame pixels it read.
__global__ void __launch_bounds__(256)
warp_backward_kernel(const float *__restrict__ mv, int W, int H, const float *__restrict__ g,
                     float *__restrict__ grad_prev) {
    const int gx = blockIdx.x * 64 + (threadIdx.x & 63);
    const int gy = blockIdx.y * 4 + (threadIdx.x >> 6);
    if (gx >= W || gy >= H) return;
    const long long N = static_cast<long long>(W) * H;
    const long long i = static_cast<long long>(gy) * W + gx;
    const float mx = __ldg(mv + i), my = __ldg(mv + N + i);
    const float ix = fminf(fmaxf(floorf(mx), -1048576.0f), 1048576.0f);
    const float iy = fminf(fmaxf(floorf(my), -1048576.0f), 1048576.0f);
    float fx = mx - floorf(mx), fy = my - floorf(my);
    int X0 = gx + static_cast<int>(ix), Y0 = gy + static_cast<int>(iy);
    if (X0 < 0) { X0 = 0; fx = 0.0f; } else if (X0 >= W - 1) { X0 = W - 1; fx = 0.0f; }
    if (Y0 < 0) { Y0 = 0; fy = 0.0f; } else if (Y0 >= H - 1) { Y0 = H - 1; fy = 0.0f; }
    const int X1 = X0 + 1 < W ? X0 + 1 : W - 1;
    const int Y1 = Y0 + 1 < H ? Y0 + 1 : H - 1;
    const long long r0 = static_cast<long long>(Y0) * W, r1 = static_cast<long long>(Y1) * W;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float v = __ldg(g + c * N + i);
        if (v == 0.0f) continue;
        float *P = grad_prev + c * N;
        atomicAdd(P + r0 + X0, (1.0f - fy) * (1.0f - fx) * v);
        atomicAdd(P + r0 + X1, (1.0f - fy) * fx * v);
        atomicAdd(P + r1 + X0, fy * (1.0f - fx) * v);
        atomicAdd(P + r1 + X1, fy * fx * v);
    }
}

__device__ __forceinline__ float tau_prime(float x, float s, float h) {
    if (x < s - 1.0f) return 0.5f * expf((x + 1.0f - s) / s);
    if (x < 1.0f - h) return 0.5f;
    return 0.5f * expf(-(x + h - 1.0f) / h);
}

__device__ __forceinline__ float tau_exact(float x, float s, float h) {
    if (x < s - 1.0f) return 0.5f * s * expf((x + 1.0f - s) / s);
    if (x < 1.0f - h) return 0.5f * (1.0f + x);
    return 1.0f - 0.5f * h * expf(-(x + h - 1.0f) / h);
}

__device__ __forceinline__ float srgb_prime(float v) {
    return v <= 0.0031308f ? 12.92f : (1.055f / 2.4f) * powf(v, 1.0f / 2.4f - 1.0f);
}

// Sec. 5 backward: grad_hdr += d sRGB(tau(x)) / d hdr applied to grad_ldr.
__global__ void __launch_bounds__(256)
tonemap_backward_kernel(const float *__restrict__ hdr, long long N, ToneArgs tm,
                        const float *__restrict__ gl, float *__restrict__ gh) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float v[3], l[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[c] = hdr[c * N + i];
        l[c] = logf(fmaxf(v[c], 0x1p-24f));
    }
    const float mean = (l[0] + l[1] + l[2]) * (1.0f / 3.0f);
    float gx[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float x = tm.alpha * (mean + tm.beta * (l[c] - mean) + tm.k);
        gx[c] = gl[c * N + i] * srgb_prime(tau_exact(x, tm.s, tm.h)) * tau_prime(x, tm.s, tm.h);
    }
    const float gs = gx[0] + gx[1] + gx[2];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float glog = tm.alpha * (tm.beta * gx[j] + (1.0f - tm.beta) * (1.0f / 3.0f) * gs);
        if (v[j] >= 0x1p-24f) gh[j * N + i] += glog / v[j];
    }
}

// Mean absolute error and its gradient sign(ldr - ref) / n.
__global__ void __launch_bounds__(256)
l1_loss_kernel(const float *__restrict__ a, const float *__restrict__ b, long long n,
               float *__restrict__ loss, float *__restrict__ grad) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    float v = 0.0f;
    if (i < n) {
        const float d = a[i] - b[i];
        v = fabsf(d);
        if (grad) grad[i] = (d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f)) / static_cast<float>(n);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __shared__ float part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < 8; ++w) t += part[w];
        atomicAdd(loss, t / static_cast<float>(n));
    }
}

// Eq. loss_combined: mean over elements of max(wt |dI - dI_ref|, ws |I - I_ref|)
// with dI = I - Wprev, dI_ref = I_ref - Wref (warped previous frames), and
// its gradient with respect to I (ties go to the spatial term).
__global__ void combined_loss_kernel(const float *__restrict__ I, const float *__restrict__ R,
                                     const float *__restrict__ P, const float *__restrict__ Q,
                                     long long n, float w, float ws,
                                     float *__restrict__ loss, float *__restrict__ grad) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    float v = 0.0f;
    if (i < n) {
        const float ds = I[i] - R[i];
        const float dt = (I[i] - P[i]) - (R[i] - Q[i]);
        const float s = ws * fabsf(ds), t = w * fabsf(dt);
        const bool temporal = t > s;
        v = temporal ? t : s;
        if (grad) {
            const float sg = temporal ? (dt > 0.0f ? w : (dt < 0.0f ? -w : 0.0f))
                                      : (ds > 0.0f ? ws : (ds < 0.0f ? -ws : 0.0f));
            grad[i] = sg / static_cast<float>(n);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __shared__ float part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int k = 0; k < 8; ++k) t += part[k];
        atomicAdd(loss, t / static_cast<float>(n));
    }
}

// Mean squared difference (for PSNR); partial sums in FP64, one atomic per block.
__global__ void sq_err_kernel(const float *__restrict__ a, const float *__restrict__ b, long long n,
                              double *__restrict__ out) {
    double v = 0.0;
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const double d = static_cast<double>(a[i]) - static_cast<double>(b[i]);
        v += d * d;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    __shared__ double part[8];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += part[w];
        atomicAdd(out, t / static_cast<double>(n));
    }
}

// Eq. app-pyramid backward: grad_L0 += 4^-l grad_L^l at the parent cell.
struct GradLayers {
    const float *p[5];
};

__global__ void __launch_bounds__(256)
pyramid_backward_kernel(GradLayers gl, int W, int H, int L, float *__restrict__ g0) {
    const int x = blockIdx.x * 64 + (threadIdx.x & 63);
    const int y = blockIdx.y * 4 + (threadIdx.x >> 6);
    if (x >= W || y >= H) return;
    const long long N = static_cast<long long>(W) * H;
    const long long i = static_cast<long long>(y) * W + x;
    float a[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int l = 1; l < 5; ++l) {
        if (l >= L) break;
        const int Wl = W >> l, Hl = H >> l;
        const long long Nl = static_cast<long long>(Wl) * Hl;
        const long long q = static_cast<long long>(y >> l) * Wl + (x >> l);
        const float sc = 1.0f / static_cast<float>(1 << (2 * l));
#pragma unroll
        for (int c = 0; c < 3; ++c) a[c] = fmaf(sc, __ldg(gl.p[l] + c * Nl + q), a[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) g0[c * N + i] += a[c];
}

// Splat backward with respect to s (Eq. stoch_rnoisy, Eq. relaxed_holdout):
//   grad_s_i = sum_c g_ic (-L0_ic / s_i)
//            + [extra, linear ramp] sum_c g_ic S_i,last,c / s_i * h lam (1 - u_i) / p_i^2
__global__ void __launch_bounds__(256)
splat_backward_kernel(const int32_t *__restrict__ offsets, const int32_t *__restrict__ counts,
                      const float4 *__restrict__ rgb, const float *__restrict__ s,
                      const float *__restrict__ L0, const float *__restrict__ gL0, long long N,
                      long long capacity, uint64_t key, float lam, float h, int hard,
                      float *__restrict__ grad_s) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float si = s[i];
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) acc -= gL0[c * N + i] * L0[c * N + i] / si;
    if (!hard) {
        const float f = floorf(si);
        const float p = si - f;
        const int n = counts[i];
        const bool extra = n > static_cast<int>(f) && p > 0.0f;
        const long long last = static_cast<long long>(offsets[i]) + n - 1;
        if (extra && last >= 0 && last < capacity) {
            const uint64_t bits = stream_bits(key, static_cast<uint64_t>(i));
            const float u = static_cast<float>(static_cast<double>(bits >> 16) * 0x1p-48);
            const float r = lam / p * (u + p - 1.0f);
            if (r > 0.0f && r < 1.0f) {
                const float dw = h * lam * (1.0f - u) / (p * p);
                const float4 S = rgb[last];
                acc += (gL0[i] * S.x + gL0[N + i] * S.y + gL0[2 * N + i] * S.z) * dw / si;
            }
        }
    }
    grad_s[i] = acc;
}

// Straight-through (estimator 1) and Gumbel-softmax (estimator 2) gradients
// of the splat with respect to s; see spp_splat_backward_estimator.
__global__ void __launch_bounds__(256)
splat_backward_est_kernel(const int32_t *__restrict__ offsets, const int32_t *__restrict__ counts,
                          const float4 *__restrict__ rgb, const float *__restrict__ s,
                          const float *__restrict__ L0, const float *__restrict__ gL0,
                          const float *__restrict__ hw, long long N, long long capacity,
                          int estimator, float lam, const float *__restrict__ clean,
                          uint64_t render_key, float *__restrict__ grad_s) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float si = s[i];
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) acc -= gL0[c * N + i] * L0[c * N + i] / si;
    const float f = floorf(si);
    const float p = si - f;
    const int n = counts[i];
    const bool extra = n > static_cast<int>(f) && p > 0.0f;
    const long long last = static_cast<long long>(offsets[i]) + n - 1;
    float3 S = make_float3(0.f, 0.f, 0.f);
    float scale = 0.0f;
    if (estimator == 2) {
        if (extra && last >= 0 && last < capacity) {
            const float w = hw[i];
            scale = lam * w * (1.0f - w) / (p * (1.0f - p));
            const float4 v = rgb[last];
            S = make_float3(v.x, v.y, v.z);
        }
    } else if (p > 0.0f) {
        scale = 1.0f;
        if (extra && last >= 0 && last < capacity) {
            const float4 v = rgb[last];
            S = make_float3(v.x, v.y, v.z);
        } else {  // the sample of slot f, which the forward did not trace
            const float g = render_factor(render_key, static_cast<uint64_t>(i),
                                          static_cast<uint64_t>(f));
            S = make_float3(clean[i] * g, clean[N + i] * g, clean[2 * N + i] * g);
        }
    }
    if (scale != 0.0f)
        acc += (gL0[i] * S.x + gL0[N + i] * S.y + gL0[2 * N + i] * S.z) * scale / si;
    grad_s[i] = acc;
}

// The DASR surrogate (Sec. 4.1, Eq. kuz_grad): (ref - L0) / n dotted with
// the loss gradient where the pixel has n >= 1 samples, ref dotted with it
// where it has none.
__global__ void __launch_bounds__(256)
splat_backward_dasr_kernel(const int32_t *__restrict__ counts, const float *__restrict__ L0,
                           const float *__restrict__ gL0, const float *__restrict__ ref,
                           long long N, float *__restrict__ grad_s) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n = counts[i];
    float acc = 0.0f;
    if (n >= 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) acc = fmaf(gL0[c * N + i], ref[c * N + i] - L0[c * N + i], acc);
        acc /= static_cast<float>(n);
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) acc = fmaf(gL0[c * N + i], ref[c * N + i], acc);
    }
    grad_s[i] = acc;
}

// Density backward, pass 1: per block, sum d and sum d g (FP64), written to
// the block's own slot; pass 1b adds the slots in index order.  No atomics:
// the sums, and the gradient, are the same from run to run.
constexpr int kDensityMaxBlocks = 2048;

__global__ void __launch_bounds__(256)
density_reduce_kernel(const float *__restrict__ d, const float *__restrict__ g, long long N,
                      double *__restrict__ partial) {
    double a = 0.0, b = 0.0;
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float di = d[i];
        a += di;
        b += static_cast<double>(di) * g[i];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    __shared__ double pa[8], pb[8];
    if ((threadIdx.x & 31) == 0) {
        pa[threadIdx.x >> 5] = a;
        pb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < 8; ++w) {
            ta += pa[w];
            tb += pb[w];
        }
        partial[2 * blockIdx.x] = ta;
        partial[2 * blockIdx.x + 1] = tb;
    }
}

__global__ void __launch_bounds__(256)
density_sum_kernel(const double *__restrict__ partial, int blocks, double *__restrict__ sums) {
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < blocks; k += blockDim.x) {
        a += partial[2 * k];
        b += partial[2 * k + 1];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    __shared__ double pa[8], pb[8];
    if ((threadIdx.x & 31) == 0) {
        pa[threadIdx.x >> 5] = a;
        pb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < 8; ++w) {
            ta += pa[w];
            tb += pb[w];
        }
        sums[0] = ta;
        sums[1] = tb;
    }
}

// Pass 2 (Sec. 3): dLoss/dz_j = (1 - phi) B N pi_j (g_j - sum_i pi_i g_i).
__global__ void __launch_bounds__(256)
density_grad_kernel(const float *__restrict__ d, const float *__restrict__ g, long long N,
                    const double *__restrict__ sums, double K, float *__restrict__ gz) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double S = sums[0];
    const double dot = sums[1] / S;
    const double pi = static_cast<double>(d[i]) / S;
    gz[i] = static_cast<float>(K * pi * (static_cast<double>(g[i]) - dot));
}

ToneArgs tone_args_bwd(const spp_tonemap *tm) {
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

template <bool UP, bool TEMP>
int launch_recon_backward(dim3 grid, dim3 block, cudaStream_t stream, const float *noisy,
                          const float *logits, int C, const float *coarse, const float *warped,
                          const uint8_t *mask, int Wl, int Hl, const float *g, float *grad_logits,
                          float *grad_noisy, float *grad_coarse, float *grad_warped) {
    constexpr int kSmem = static_cast<int>(sizeof(BwdSmem<UP, TEMP>));
    static int configured_dev = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPP_ERR_CUDA;
    if (configured_dev != dev) {
        if (cudaFuncSetAttribute(recon_backward_kernel<UP, TEMP>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem) != cudaSuccess)
            return SPP_ERR_CUDA;
        configured_dev = dev;
    }
    recon_backward_kernel<UP, TEMP><<<grid, block, kSmem, stream>>>(
        noisy, logits, C, coarse, warped, mask, Wl, Hl, g, grad_logits, grad_noisy, grad_coarse,
        grad_warped);
    return SPP_OK;
}

}  // namespace
}  // namespace spp

extern "C" {

int spp_reconstruct_level_backward(const float *noisy, const float *logits, int C,
                                   const float *coarse, const float *warped_prev,
                                   const uint8_t *mask, int Wl, int Hl, const float *grad_out,
                                   float *grad_logits, float *grad_noisy, float *grad_coarse,
                                   float *grad_warped, cudaStream_t stream) {
    using namespace spp;
    if (Wl < 0 || Hl < 0 || !noisy || !logits || !grad_out || !grad_logits) return SPP_ERR_ARG;
    if (warped_prev && !coarse) return SPP_ERR_ARG;
    const int need = 25 + (coarse ? 4 : 0);
    if (C < need || (warped_prev && C < 54)) return SPP_ERR_ARG;
    if (coarse && ((Wl & 1) || (Hl & 1))) return SPP_ERR_SHAPE;
    if (!aligned16(noisy) || !aligned16(logits) || !aligned16(grad_out) ||
        !aligned16(grad_logits) || (coarse && !aligned16(coarse)) ||
        (warped_prev && !aligned16(warped_prev)) || (mask && !aligned16(mask)) ||
        (grad_noisy && !aligned16(grad_noisy)) || (grad_coarse && !aligned16(grad_coarse)) ||
        (grad_warped && !aligned16(grad_warped)))
        return SPP_ERR_ALIGN;
    if (static_cast<long long>(Wl) * Hl == 0) return SPP_OK;
    dim3 block(kBX, kBY);
    dim3 grid((Wl + kBX - 1) / kBX, (Hl + kBY - 1) / kBY);
    int rc;
    if (!coarse)
        rc = launch_recon_backward<false, false>(grid, block, stream, noisy, logits, C, coarse,
                                                 warped_prev, mask, Wl, Hl, grad_out, grad_logits,
                                                 grad_noisy, grad_coarse, grad_warped);
    else if (!warped_prev)
        rc = launch_recon_backward<true, false>(grid, block, stream, noisy, logits, C, coarse,
                                                warped_prev, mask, Wl, Hl, grad_out, grad_logits,
                                                grad_noisy, grad_coarse, grad_warped);
    else
        rc = launch_recon_backward<true, true>(grid, block, stream, noisy, logits, C, coarse,
                                               warped_prev, mask, Wl, Hl, grad_out, grad_logits,
                                               grad_noisy, grad_coarse, grad_warped);
    count_launch();
    return rc != SPP_OK ? rc : launch_status();
}

int spp_warp_previous_backward(const float *mv, int W, int H, const float *grad_warped,
                               float *grad_prev, cudaStream_t stream) {
    using namespace spp;
    if (W < 0 || H < 0 || !mv || !grad_warped || !grad_prev) return SPP_ERR_ARG;
    if (!aligned16(mv) || !aligned16(grad_warped) || !aligned16(grad_prev)) return SPP_ERR_ALIGN;
    if (static_cast<long long>(W) * H == 0) return SPP_OK;
    dim3 grid((W + 63) / 64, (H + 3) / 4);
    warp_backward_kernel<<<grid, 256, 0, stream>>>(mv, W, H, grad_warped, grad_prev);
    count_launch();
    return launch_status();
}

int spp_tonemap_backward(const float *hdr, int W, int H, const spp_tonemap *tm,
                         const float *grad_ldr, float *grad_hdr, cudaStream_t stream) {
    using namespace spp;
    if (W < 0 || H < 0 || !hdr || !grad_ldr || !grad_hdr) return SPP_ERR_ARG;
    if (!aligned16(hdr) || !aligned16(grad_ldr) || !aligned16(grad_hdr)) return SPP_ERR_ALIGN;
    const ToneArgs ta = tone_args_bwd(tm);
    if (!(ta.s > 0.0f && ta.s < 1.0f && ta.h > 0.0f && ta.h < 1.0f)) return SPP_ERR_ARG;
    const long long N = static_cast<long long>(W) * H;
    if (N == 0) return SPP_OK;
    tonemap_backward_kernel<<<static_cast<unsigned>((N + 255) / 256), 256, 0, stream>>>(
        hdr, N, ta, grad_ldr, grad_hdr);
    count_launch();
    return launch_status();
}

int spp_l1_loss(const float *ldr, const float *ref, int64_t n, float *loss, float *grad_ldr,
                cudaStream_t stream) {
    using namespace spp;
    if (n < 0 || !ldr || !ref || !loss) return SPP_ERR_ARG;
    if (!aligned16(ldr) || !aligned16(ref) || (grad_ldr && !aligned16(grad_ldr)) || !aligned16(loss))
        return SPP_ERR_ALIGN;
    if (cudaMemsetAsync(loss, 0, sizeof(float), stream) != cudaSuccess) return SPP_ERR_CUDA;
    if (n == 0) return SPP_OK;
    l1_loss_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(
        ldr, ref, static_cast<long long>(n), loss, grad_ldr);
    count_launch();
    return launch_status();
}

int spp_combined_loss(const float *ldr, const float *ref, const float *prev_warped,
                      const float *ref_prev_warped, int64_t n, float temporal_weight,
                      float spatial_weight, float *loss, float *grad_ldr, cudaStream_t stream) {
    using namespace spp;
    if (n < 0 || !ldr || !ref || !prev_warped || !ref_prev_warped || !loss) return SPP_ERR_ARG;
    if (!aligned16(ldr) || !aligned16(ref) || !aligned16(prev_warped) ||
        !aligned16(ref_prev_warped) || !aligned16(loss) || (grad_ldr && !aligned16(grad_ldr)))
        return SPP_ERR_ALIGN;
    if (cudaMemsetAsync(loss, 0, sizeof(float), stream) != cudaSuccess) return SPP_ERR_CUDA;
    if (n == 0) return SPP_OK;
    combined_loss_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, stream>>>(
        ldr, ref, prev_warped, ref_prev_warped, static_cast<long long>(n), temporal_weight,
        spatial_weight, loss, grad_ldr);
    count_launch();
    return launch_status();
}

int spp_mse(const float *a, const float *b, int64_t n, double *mse, cudaStream_t stream) {
    using namespace spp;
    if (n < 0 || !a || !b || !mse) return SPP_ERR_ARG;
    if (!aligned16(a) || !aligned16(b) || !aligned16(mse)) return SPP_ERR_ALIGN;
    if (cudaMemsetAsync(mse, 0, sizeof(double), stream) != cudaSuccess) return SPP_ERR_CUDA;
    if (n == 0) return SPP_OK;
    const long long blocks = std::min<long long>((n + 255) / 256, 4LL * sm_count());
    sq_err_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(a, b, n, mse);
    count_launch();
    return launch_status();
}

int spp_pyramid_backward(const float *const *grad_layers, int W, int H, int L, float *grad_L0,
                         cudaStream_t stream) {
    using namespace spp;
    if (W < 0 || H < 0 || !grad_layers || !grad_L0) return SPP_ERR_ARG;
    if (L < 1 || L > 5) return SPP_ERR_SHAPE;
    if ((W % (1 << (L - 1))) != 0 || (H % (1 << (L - 1))) != 0) return SPP_ERR_SHAPE;
    GradLayers gl{};
    for (int l = 1; l < L; ++l) {
        if (!grad_layers[l]) return SPP_ERR_ARG;
        if (!aligned16(grad_layers[l])) return SPP_ERR_ALIGN;
        gl.p[l] = grad_layers[l];
    }
    if (!aligned16(grad_L0)) return SPP_ERR_ALIGN;
    if (static_cast<long long>(W) * H == 0 || L == 1) return SPP_OK;
    dim3 grid((W + 63) / 64, (H + 3) / 4);
    pyramid_backward_kernel<<<grid, 256, 0, stream>>>(gl, W, H, L, grad_L0);
    count_launch();
    return launch_status();
}

int spp_splat_backward(const int32_t *offsets, const int32_t *counts, const float *rgb,
                       const float *s, const float *layer0, const float *grad_layer0,
                       int64_t capacity, int W, int H, const spp_params *p, float *grad_s,
                       cudaStream_t stream) {
    using namespace spp;
    if (W < 0 || H < 0 || capacity < 0 || !p || !offsets || !counts || !s || !layer0 ||
        !grad_layer0 || !grad_s || (capacity > 0 && !rgb))
        return SPP_ERR_ARG;
    if (!aligned16(offsets) || !aligned16(counts) || (rgb && !aligned16(rgb)) || !aligned16(s) ||
        !aligned16(layer0) || !aligned16(grad_layer0) || !aligned16(grad_s))
        return SPP_ERR_ALIGN;
    const long long N = static_cast<long long>(W) * H;
    if (N == 0) return SPP_OK;
    const bool hard = p->holdout_mode == SPP_HOLDOUT_HARD;
    const double lam = hard ? 1.0 : p->lambda;
    const double h = 2.0 * lam / (2.0 * lam - 1.0);
    splat_backward_kernel<<<static_cast<unsigned>((N + 255) / 256), 256, 0, stream>>>(
        offsets, counts, reinterpret_cast<const float4 *>(rgb), s, layer0, grad_layer0, N, capacity,
        stream_key(p->seed, p->frame), static_cast<float>(lam), static_cast<float>(h), hard ? 1 : 0,
        grad_s);
    count_launch();
    return launch_status();
}

int spp_splat_backward_estimator(const int32_t *offsets, const int32_t *counts, const float *rgb,
                                 const float *s, const float *layer0, const float *grad_layer0,
                                 const float *holdout_w, int64_t capacity, int W, int H,
                                 const spp_params *p, int estimator, const float *clean,
                                 uint64_t render_seed, float *grad_s, cudaStream_t stream) {
    using namespace spp;
    if (estimator == SPP_ESTIMATOR_RELAXED)
        return spp_splat_backward(offsets, counts, rgb, s, layer0, grad_layer0, capacity, W, H, p,
                                  grad_s, stream);
    if (estimator == SPP_ESTIMATOR_DASR) {
        if (W < 0 || H < 0 || !counts || !layer0 || !grad_layer0 || !clean || !grad_s)
            return SPP_ERR_ARG;
        if (!aligned16(counts) || !aligned16(layer0) || !aligned16(grad_layer0) ||
            !aligned16(clean) || !aligned16(grad_s))
            return SPP_ERR_ALIGN;
        const long long N = static_cast<long long>(W) * H;
        if (N == 0) return SPP_OK;
        splat_backward_dasr_kernel<<<static_cast<unsigned>((N + 255) / 256), 256, 0, stream>>>(
            counts, layer0, grad_layer0, clean, N, grad_s);
        count_launch();
        return launch_status();
    }
    if (estimator != SPP_ESTIMATOR_STRAIGHT_THROUGH && estimator != SPP_ESTIMATOR_GUMBEL)
        return SPP_ERR_ARG;
    if (!p || W < 0 || H < 0 || capacity < 0 || !offsets || !counts || !s || !layer0 ||
        !grad_layer0 || !grad_s || (capacity > 0 && !rgb))
        return SPP_ERR_ARG;
    if (estimator == SPP_ESTIMATOR_GUMBEL && (!holdout_w || !(p->lambda > 0.0)))
        return SPP_ERR_ARG;
    if (estimator == SPP_ESTIMATOR_STRAIGHT_THROUGH && !clean) return SPP_ERR_ARG;
    if (!aligned16(offsets) || !aligned16(counts) || !aligned16(s) || !aligned16(layer0) ||
        !aligned16(grad_layer0) || !aligned16(grad_s) || (rgb && !aligned16(rgb)) ||
        (holdout_w && !aligned16(holdout_w)) || (clean && !aligned16(clean)))
        return SPP_ERR_ALIGN;
    const long long N = static_cast<long long>(W) * H;
    if (N == 0) return SPP_OK;
    splat_backward_est_kernel<<<static_cast<unsigned>((N + 255) / 256), 256, 0, stream>>>(
        offsets, counts, reinterpret_cast<const float4 *>(rgb), s, layer0, grad_layer0, holdout_w,
        N, capacity, estimator, static_cast<float>(p->lambda), clean,
        stream_key(render_seed, p->frame), grad_s);
    count_launch();
    return launch_status();
}

size_t spp_density_backward_workspace_bytes(void) {
    return 256 + static_cast<size_t>(spp::kDensityMaxBlocks) * 2 * sizeof(double);
}

int spp_density_backward(const float *d, int64_t N, double budget, double uniform_fraction,
                         const float *grad_s, float *grad_z, void *ws, size_t ws_bytes,
                         cudaStream_t stream) {
    using namespace spp;
    if (N < 0 || !d || !grad_s || !grad_z || !ws) return SPP_ERR_ARG;
    if (ws_bytes < spp_density_backward_workspace_bytes()) return SPP_ERR_WORKSPACE;
    if (!aligned16(d) || !aligned16(grad_s) || !aligned16(grad_z) || !aligned16(ws))
        return SPP_ERR_ALIGN;
    if (N == 0) return SPP_OK;
    double *sums = static_cast<double *>(ws);
    double *partial = reinterpret_cast<double *>(static_cast<unsigned char *>(ws) + 256);
    long long blocks = (N + 255) / 256;
    long long rblocks = static_cast<long long>(sm_count()) * 8;
    if (rblocks > blocks) rblocks = blocks;
    if (rblocks > kDensityMaxBlocks) rblocks = kDensityMaxBlocks;
    density_reduce_kernel<<<static_cast<unsigned>(rblocks), 256, 0, stream>>>(d, grad_s, N,
                                                                           partial);
    density_sum_kernel<<<1, 256, 0, stream>>>(partial, static_cast<int>(rblocks), sums);
    const double K = (1.0 - uniform_fraction) * budget * static_cast<double>(N);
    density_grad_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(d, grad_s, N, sums, K,
                                                                           grad_z);
    count_launch(3);
    return launch_status();
}

}  // extern "C"
