// a11: backward pass of the sampling + reconstruction path (arXiv 2602.08642):
// the joint-softmax gather pyramid (App. A), the reprojection W_t, the tone
// map (Sec. 5), the L1 loss in sRGB (Eq. loss_spatial with m = 1), the
// average-pool pyramid, the density-normalised splat with the relaxed ramp
// (Eq. stoch_rnoisy, Eq. relaxed_holdout) and the spatial softmax of the
// sampler output (Sec. 3).
//
// The reconstruction backward recomputes each pixel's softmax weights from
// its logits instead of storing the K x K tap products.  Gradients that
// scatter to neighbouring pixels (the gather taps, the bilinear warp) are
// summed in shared memory over the block's tile and halo first and then
// added to global memory with atomics, so their summation order (and the
// last bits of those gradients) may vary from run to run.
#include "recon_common.cuh"
#include "render_common.cuh"

namespace spp {
namespace {

constexpr int kBX = 32, kBY = 8, kBH = 2;
constexpr int kBHX = kBX + 2 * kBH, kBHY = kBY + 2 * kBH;
constexpr int kCX = kBX / 2 + 1, kCY = kBY / 2 + 1;  // coarse footprint of a tile

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
    __shared__ float sN[3][kBHY][kBHX];
    __shared__ float sW[TEMP ? 3 : 1][TEMP ? kBHY : 1][TEMP ? kBHX : 1];
    __shared__ float aN[3][kBHY][kBHX];
    __shared__ float aW[TEMP ? 3 : 1][TEMP ? kBHY : 1][TEMP ? kBHX : 1];
    __shared__ float aC[UP ? 3 : 1][UP ? kCY : 1][UP ? kCX : 1];

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kBX + tx;
    const int bx0 = blockIdx.x * kBX, by0 = blockIdx.y * kBY;
    const int x = bx0 + tx, y = by0 + ty;
    const bool inside = x < Wl && y < Hl;
    const int xc = min(x, Wl - 1), yc = min(y, Hl - 1);
    const long long Nl = static_cast<long long>(Wl) * Hl;
    const long long pix = static_cast<long long>(yc) * Wl + xc;
    const int Wc = Wl >> 1, Hc = Hl >> 1;
    const long long Nc = static_cast<long long>(Wc) * Hc;
    const int cbx = bx0 >> 1, cby = by0 >> 1;  // first coarse cell of the footprint

    for (int idx = tid; idx < kBHX * kBHY; idx += kBX * kBY) {
        const int hx = idx % kBHX, hy = idx / kBHX;
        const int gx = clampi(bx0 + hx - kBH, 0, Wl - 1), gy = clampi(by0 + hy - kBH, 0, Hl - 1);
        const long long q = static_cast<long long>(gy) * Wl + gx;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sN[c][hy][hx] = __ldg(noisy + c * Nl + q);
            aN[c][hy][hx] = 0.0f;
            if (TEMP) {
                sW[c][hy][hx] = __ldg(warped + c * Nl + q);
                aW[c][hy][hx] = 0.0f;
            }
        }
    }
    if (UP)
        for (int idx = tid; idx < kCX * kCY; idx += kBX * kBY)
#pragma unroll
            for (int c = 0; c < 3; ++c) aC[c][idx / kCX][idx % kCX] = 0.0f;
    __syncthreads();

    // recompute the joint softmax of this pixel
    float lg[kNK];
#pragma unroll
    for (int k = 0; k < kSpatial; ++k) lg[k] = __ldg(logits + k * Nl + pix);
    const bool use_t = TEMP && !(mask && mask[pix]);
    if (TEMP) {
#pragma unroll
        for (int k = 0; k < 25; ++k) lg[kSpatial + k] = use_t ? __ldg(logits + (29 + k) * Nl + pix) : 0.0f;
    }
    float m = lg[0];
#pragma unroll
    for (int k = 1; k < kSpatial; ++k) m = fmaxf(m, lg[k]);
    if (use_t) {
#pragma unroll
        for (int k = kSpatial; k < kNK; ++k) m = fmaxf(m, lg[k]);
    }
    float wsum = 0.0f;
#pragma unroll
    for (int k = 0; k < kNK; ++k) {
        const bool on = k < kSpatial || use_t;
        lg[k] = on ? __expf(lg[k] - m) : 0.0f;  // lg now holds the unnormalised weights
        wsum += lg[k];
    }
    const float inv = 1.0f / wsum;
    const float g0 = inside ? __ldg(g + pix) : 0.0f;
    const float g1 = inside ? __ldg(g + Nl + pix) : 0.0f;
    const float g2 = inside ? __ldg(g + 2 * Nl + pix) : 0.0f;

    // tap values and q_k = sum_c g_c v_kc
    float q[kNK];
    float cvv[UP ? 12 : 1];
    int cidx[UP ? 4 : 1];
#pragma unroll
    for (int j = 0; j < 5; ++j)
#pragma unroll
        for (int i = 0; i < 5; ++i)
            q[j * 5 + i] = g0 * sN[0][ty + j][tx + i] + g1 * sN[1][ty + j][tx + i] +
                           g2 * sN[2][ty + j][tx + i];
    if (UP) {
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int cx = min((xc + i) >> 1, Wc - 1), cy = min((yc + j) >> 1, Hc - 1);
                const long long qq = static_cast<long long>(cy) * Wc + cx;
                const int t = 2 * j + i;
                cidx[t] = (cy - cby) * kCX + (cx - cbx);
                cvv[3 * t] = __ldg(coarse + qq);
                cvv[3 * t + 1] = __ldg(coarse + Nc + qq);
                cvv[3 * t + 2] = __ldg(coarse + 2 * Nc + qq);
                q[25 + t] = g0 * cvv[3 * t] + g1 * cvv[3 * t + 1] + g2 * cvv[3 * t + 2];
            }
    }
    if (TEMP) {
#pragma unroll
        for (int j = 0; j < 5; ++j)
#pragma unroll
            for (int i = 0; i < 5; ++i)
                q[kSpatial + j * 5 + i] = g0 * sW[0][ty + j][tx + i] + g1 * sW[1][ty + j][tx + i] +
                                          g2 * sW[2][ty + j][tx + i];
    }
    float qbar = 0.0f;
#pragma unroll
    for (int k = 0; k < kNK; ++k) qbar = fmaf(lg[k] * inv, q[k], qbar);

    if (inside) {
        // dLoss/dz_k = w_k (q_k - qbar); channels without a kernel get 0
#pragma unroll
        for (int k = 0; k < kSpatial; ++k) grad_logits[k * Nl + pix] = lg[k] * inv * (q[k] - qbar);
        if (TEMP) {
#pragma unroll
            for (int k = 0; k < 25; ++k)
                grad_logits[(29 + k) * Nl + pix] =
                    use_t ? lg[kSpatial + k] * inv * (q[kSpatial + k] - qbar) : 0.0f;
        }
        for (int k = TEMP ? 54 : kSpatial; k < C; ++k) grad_logits[k * Nl + pix] = 0.0f;
        // dLoss/dv_kc = w_k g_c, summed per source cell in shared memory
#pragma unroll
        for (int j = 0; j < 5; ++j)
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                const float w = lg[j * 5 + i] * inv;
                atomicAdd(&aN[0][ty + j][tx + i], w * g0);
                atomicAdd(&aN[1][ty + j][tx + i], w * g1);
                atomicAdd(&aN[2][ty + j][tx + i], w * g2);
            }
        if (UP) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float w = lg[25 + t] * inv;
                float *a = &aC[0][0][0];
                atomicAdd(a + cidx[t], w * g0);
                atomicAdd(a + kCX * kCY + cidx[t], w * g1);
                atomicAdd(a + 2 * kCX * kCY + cidx[t], w * g2);
            }
        }
        if (use_t) {
#pragma unroll
            for (int j = 0; j < 5; ++j)
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    const float w = lg[kSpatial + j * 5 + i] * inv;
                    atomicAdd(&aW[0][ty + j][tx + i], w * g0);
                    atomicAdd(&aW[1][ty + j][tx + i], w * g1);
                    atomicAdd(&aW[2][ty + j][tx + i], w * g2);
                }
        }
    }
    __syncthreads();
    // halo cells beyond the image hold the clamped pixels' contributions:
    // adding them at the clamped coordinate is the clamp-to-edge transpose
    for (int idx = tid; idx < kBHX * kBHY; idx += kBX * kBY) {
        const int hx = idx % kBHX, hy = idx / kBHX;
        const int gx = clampi(bx0 + hx - kBH, 0, Wl - 1), gy = clampi(by0 + hy - kBH, 0, Hl - 1);
        const long long qq = static_cast<long long>(gy) * Wl + gx;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = aN[c][hy][hx];
            if (v != 0.0f && grad_noisy) atomicAdd(grad_noisy + c * Nl + qq, v);
            if (TEMP) {
                const float vw = aW[c][hy][hx];
                if (vw != 0.0f && grad_warped) atomicAdd(grad_warped + c * Nl + qq, vw);
            }
        }
    }
    if (UP && grad_coarse)
        for (int idx = tid; idx < kCX * kCY; idx += kBX * kBY) {
            const int cx = cbx + idx % kCX, cy = cby + idx / kCX;
            if (cx >= Wc || cy >= Hc) continue;
            const long long qq = static_cast<long long>(cy) * Wc + cx;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float v = aC[c][idx / kCX][idx % kCX];
                if (v != 0.0f) atomicAdd(grad_coarse + c * Nc + qq, v);
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

// Density backward, pass 1: sum d and sum d g (FP64 accumulation).
__global__ void __launch_bounds__(256)
density_reduce_kernel(const float *__restrict__ d, const float *__restrict__ g, long long N,
                      double *__restrict__ sums) {
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
        atomicAdd(sums, ta);
        atomicAdd(sums + 1, tb);
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
    if (!coarse)
        recon_backward_kernel<false, false><<<grid, block, 0, stream>>>(
            noisy, logits, C, coarse, warped_prev, mask, Wl, Hl, grad_out, grad_logits, grad_noisy,
            grad_coarse, grad_warped);
    else if (!warped_prev)
        recon_backward_kernel<true, false><<<grid, block, 0, stream>>>(
            noisy, logits, C, coarse, warped_prev, mask, Wl, Hl, grad_out, grad_logits, grad_noisy,
            grad_coarse, grad_warped);
    else
        recon_backward_kernel<true, true><<<grid, block, 0, stream>>>(
            noisy, logits, C, coarse, warped_prev, mask, Wl, Hl, grad_out, grad_logits, grad_noisy,
            grad_coarse, grad_warped);
    count_launch();
    return launch_status();
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

size_t spp_density_backward_workspace_bytes(void) { return 256; }

int spp_density_backward(const float *d, int64_t N, double budget, double uniform_fraction,
                         const float *grad_s, float *grad_z, void *ws, size_t ws_bytes,
                         cudaStream_t stream) {
    using namespace spp;
    if (N < 0 || !d || !grad_s || !grad_z || !ws) return SPP_ERR_ARG;
    if (ws_bytes < spp_density_backward_workspace_bytes()) return SPP_ERR_WORKSPACE;
    if (!aligned16(d) || !aligned16(grad_s) || !aligned16(grad_z) || !aligned16(ws))
        return SPP_ERR_ALIGN;
    if (N == 0) return SPP_OK;
    if (cudaMemsetAsync(ws, 0, 2 * sizeof(double), stream) != cudaSuccess) return SPP_ERR_CUDA;
    double *sums = static_cast<double *>(ws);
    long long blocks = (N + 255) / 256;
    const long long cap = static_cast<long long>(sm_count()) * 8;
    density_reduce_kernel<<<static_cast<unsigned>(blocks < cap ? blocks : cap), 256, 0, stream>>>(
        d, grad_s, N, sums);
    const double K = (1.0 - uniform_fraction) * budget * static_cast<double>(N);
    density_grad_kernel<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(d, grad_s, N, sums, K,
                                                                           grad_z);
    count_launch(2);
    return launch_status();
}

}  // extern "C"
