/*
 * spp_oracle.c -- plain, slow, FP64 CPU oracle for the sub-1-spp adaptive
 * sampling and gather-pyramid reconstruction path of "Forget Superresolution,
 * Sample Adaptively (when Path Tracing)" (arXiv 2602.08642).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  The product path (the CUDA
 * library) never calls it, shares no code, header, table or constant with it,
 * and fails loudly when its own extension is missing.
 *
 * Every function restates one step of the paper in plain loops, in FP64, in
 * the order the paper states it.  Compile with -ffp-contract=off so that no
 * multiply-add is fused: the count map depends on the exact FP64 rounding of
 * the budget normalisation (Sec. 3) and of the fractional part (Sec. 4.2).
 *
 * Readings of the paper where it is silent (the GPU path takes the same ones):
 *   - uniforms u_i: SplitMix64 output mix of a per-pixel counter (the
 *     paper dithers with blue noise, Sec. 6.3; white noise is used here);
 *   - extra sample iff u_i > 1 - p_i (Eq. relaxed_holdout and the test-time
 *     rule of Sec. 4.3: no sample when u_i < 1 - p_i);
 *   - the extra (holdout) sample is the last slot of its pixel;
 *   - clamp-to-edge addressing for the gather G, the upsampling U and the
 *     reprojection W_t (Appendix A is silent about borders);
 *   - upsampling taps at floor((x+i)/2), i in {0,1}, exactly as printed in
 *     Eq. app-upsample, clamped at the far edge of the coarser level;
 *   - kernel channel order: denoise tap (i,j) -> (j+2)*5 + (i+2); upsampling
 *     tap (i,j) -> 25 + 2j + i; temporal tap (i,j) -> 29 + (j+2)*5 + (i+2);
 *   - W_t: bilinear sample of the previous HDR output at (x+mv_x, y+mv_y),
 *     pixel centres at integer coordinates, position clamped to the frame;
 *   - disoccluded pixels (mask != 0) and frames without a previous output
 *     drop the 25 temporal logits from the joint softmax.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_INPUT -2

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number     */
/* generators", OOPSLA 2014): golden-gamma increment and the variant-13     */
/* output mix.                                                               */
/* ------------------------------------------------------------------------ */
static const uint64_t ORC_GOLDEN_GAMMA = 0x9E3779B97F4A7C15ULL;

/* Threads of the parallel loops (OpenMP over pixels or rows; every pixel is
 * computed alone, so the results do not depend on the count).  n <= 0
 * restores the default; without OpenMP everything runs on one thread. */
void orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

uint64_t orc_splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Sequential generator: advance the state by the golden gamma, then mix. */
uint64_t orc_splitmix64_next(uint64_t *state) {
    *state += ORC_GOLDEN_GAMMA;
    return orc_splitmix64_mix(*state);
}

/* Counter-based per-pixel bits.  One SplitMix64 stream per (seed, frame):
 *   key  = mix(seed + (frame + 1) * gamma)
 *   bits = mix(key + (i + 1) * gamma)        (64-bit wrap-around)
 * i.e. element i of the SplitMix64 sequence that starts at state key. */
uint64_t orc_stream_key(uint64_t seed, uint32_t frame) {
    return orc_splitmix64_mix(seed + ((uint64_t)frame + 1) * ORC_GOLDEN_GAMMA);
}

uint64_t orc_pixel_bits(uint64_t seed, uint32_t frame, uint64_t i) {
    uint64_t key = orc_stream_key(seed, frame);
    return orc_splitmix64_mix(key + (i + 1) * ORC_GOLDEN_GAMMA);
}

/* The discretisation uniform u_i in [0,1): the top 48 bits scaled by 2^-48
 * (exact in FP64).  Sec. 4.2 draws u_i ~ U(0,1) once per pixel. */
double orc_pixel_uniform(uint64_t seed, uint32_t frame, uint64_t i) {
    uint64_t b = orc_pixel_bits(seed, frame, i);
    return (double)(b >> 16) * 0x1p-48;
}

/* ------------------------------------------------------------------------ */
/* Exact sum of FP32 values, correctly rounded to FP64.                      */
/* Shewchuk, "Adaptive Precision Floating-Point Arithmetic and Fast Robust   */
/* Geometric Predicates" (1997): the running sum is kept as a list of        */
/* non-overlapping FP64 partials grown by error-free two-sums; the final     */
/* value is rounded once, with the half-way case settled by the sign of the  */
/* next partial.  Sec. 3 needs the sum of the sampler output for the         */
/* softmax normalisation; exact rounding makes it order-independent.         */
/* ------------------------------------------------------------------------ */
#define ORC_MAXPARTIALS 64

static double orc_round_partials(const double *part, int n) {
    if (n == 0) return 0.0;
    double hi = part[--n];
    double lo = 0.0;
    while (n > 0) {
        double x = hi;
        double y = part[--n];
        hi = x + y;
        double yr = hi - x;
        lo = y - yr;
        if (lo != 0.0) break;
    }
    /* hi + lo is exact; the remaining partials are below lo.  If lo is
     * exactly half an ulp of hi, the sign of the next partial decides. */
    if (n > 0 && ((lo < 0.0 && part[n - 1] < 0.0) || (lo > 0.0 && part[n - 1] > 0.0))) {
        double y = lo * 2.0;
        double x = hi + y;
        double yr = x - hi;
        if (y == yr) hi = x;
    }
    return hi;
}

double orc_exact_sum_f32(const float *v, int64_t n) {
    double part[ORC_MAXPARTIALS];
    int np = 0;
    for (int64_t k = 0; k < n; ++k) {
        double x = (double)v[k];
        int i = 0;
        for (int j = 0; j < np; ++j) {
            double y = part[j];
            if (fabs(x) < fabs(y)) { double t = x; x = y; y = t; }
            double hi = x + y;
            double lo = y - (hi - x);
            if (lo != 0.0) part[i++] = lo;
            x = hi;
        }
        part[i++] = x;
        np = i;
        if (np >= ORC_MAXPARTIALS) return NAN; /* cannot happen for finite FP32 input */
    }
    return orc_round_partials(part, np);
}

/* Same algorithm over FP64 inputs (used by the pins for sum(s_i) = B N). */
double orc_exact_sum_f64(const double *v, int64_t n) {
    double part[ORC_MAXPARTIALS];
    int np = 0;
    for (int64_t k = 0; k < n; ++k) {
        double x = v[k];
        int i = 0;
        for (int j = 0; j < np; ++j) {
            double y = part[j];
            if (fabs(x) < fabs(y)) { double t = x; x = y; y = t; }
            double hi = x + y;
            double lo = y - (hi - x);
            if (lo != 0.0) part[i++] = lo;
            x = hi;
        }
        part[i++] = x;
        np = i;
        if (np >= ORC_MAXPARTIALS) return NAN;
    }
    return orc_round_partials(part, np);
}

/* ------------------------------------------------------------------------ */
/* a1: budget normalisation (Sec. 3).                                        */
/* s_i = B*phi + ((1-phi) * B * N / S) * d_i with S = sum_j d_j and          */
/* phi = 1/8 in the paper.  d is the sampler's non-negative output already   */
/* exponentiated, so d_i / S is the spatial softmax.  Each operation is one  */
/* FP64 round-to-nearest step, in this order: a = phi*B;                      */
/* c = (((1-phi)*B) * N) / S; s_i = a + (c * d_i).                           */
/* ------------------------------------------------------------------------ */
int orc_budget_coeffs(const float *d, int64_t N, double B, double phi,
                      double *S_out, double *a_out, double *c_out) {
    if (N < 0 || !(B > 0.0) || !(phi >= 0.0) || !(phi <= 1.0)) return ORC_ERR_ARG;
    for (int64_t i = 0; i < N; ++i) {
        float x = d[i];
        if (!(x >= 0.0f) || isinf(x)) return ORC_ERR_INPUT; /* NaN, negative, inf */
    }
    double S = orc_exact_sum_f32(d, N);
    if (N > 0 && !(S > 0.0)) return ORC_ERR_INPUT;
    double a = phi * B;
    double k = (1.0 - phi) * B;
    double num = k * (double)N;
    double c = (N > 0) ? num / S : 0.0;
    *S_out = S;
    *a_out = a;
    *c_out = c;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* a2: stochastic rounding with the relaxed holdout ramp (Sec. 4.2, 4.3).    */
/* f = floor(s), p = s - f.  One extra sample iff p > 0 and u > 1 - p.       */
/* Its weight in the splat is the ramp of Eq. relaxed_holdout,               */
/*   H = h * min(max((lambda/p) * (u + p - 1), 0), 1),                       */
/* with h = 2 lambda / (2 lambda - 1) (Eq. h_factor).  In hard mode the      */
/* weight is 1 (the lambda -> infinity limit of Sec. 4.3).                   */
/* ------------------------------------------------------------------------ */
void orc_assign_one(double s, double u, double lambda, int hard,
                    int64_t *n_out, double *w_out, int *extra_out) {
    double f = floor(s);
    double p = s - f;
    double t = 1.0 - p;
    int extra = (p > 0.0) && (u > t);
    double w = 1.0;
    if (extra && !hard) {
        double h = (2.0 * lambda) / (2.0 * lambda - 1.0);
        double q = lambda / p;
        double v = (u + p) - 1.0;
        double r = q * v;
        if (r < 0.0) r = 0.0;
        if (r > 1.0) r = 1.0;
        w = h * r;
    }
    *n_out = (int64_t)f + extra;
    *w_out = w;
    *extra_out = extra;
}

/* Whole-frame allocation: s, counts, holdout weights and the exclusive scan
 * of the counts (the sample list's offsets; the samples of pixel i occupy
 * slots offsets[i] .. offsets[i+1]-1, the extra one last).  w_out[i] is the
 * weight of pixel i's last slot: the ramp weight when the extra sample is
 * taken, 1 otherwise. */
int orc_alloc(const float *d, int64_t N, double B, double phi, double lambda, int hard,
              uint64_t seed, uint32_t frame,
              double *s_out, int64_t *counts, int64_t *offsets, double *w_out,
              int32_t *extra_out, double *coeffs_out /* S, a, c */) {
    double S, a, c;
    int rc = orc_budget_coeffs(d, N, B, phi, &S, &a, &c);
    if (rc != ORC_OK) return rc;
    if (coeffs_out) { coeffs_out[0] = S; coeffs_out[1] = a; coeffs_out[2] = c; }
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double m = c * (double)d[i];
        double s = a + m;
        double u = orc_pixel_uniform(seed, frame, (uint64_t)i);
        int64_t n; double w; int extra;
        orc_assign_one(s, u, lambda, hard, &n, &w, &extra);
        s_out[i] = s;
        counts[i] = n;
        w_out[i] = w;
        if (extra_out) extra_out[i] = extra;
    }
    int64_t run = 0;
    for (int64_t i = 0; i < N; ++i) {
        offsets[i] = run;
        run += counts[i];
    }
    offsets[N] = run;
    return ORC_OK;
}

/* a1-a2 with explicit uniforms: u_i = u48[i] 2^-48 (the blue-noise dither of
 * Sec. 6.3 instead of the counter-based white noise); otherwise orc_alloc. */
int orc_alloc_u48(const float *d, int64_t N, double B, double phi, double lambda, int hard,
                  const uint64_t *u48, double *s_out, int64_t *counts, int64_t *offsets,
                  double *w_out, int32_t *extra_out, double *coeffs_out) {
    double S, a, c;
    int rc = orc_budget_coeffs(d, N, B, phi, &S, &a, &c);
    if (rc != ORC_OK) return rc;
    if (coeffs_out) { coeffs_out[0] = S; coeffs_out[1] = a; coeffs_out[2] = c; }
    int64_t run = 0;
    for (int64_t i = 0; i < N; ++i) {
        double m = c * (double)d[i];
        double s = a + m;
        double u = (double)u48[i] * 0x1p-48;
        int64_t n; double w; int extra;
        orc_assign_one(s, u, lambda, hard, &n, &w, &extra);
        s_out[i] = s;
        counts[i] = n;
        w_out[i] = w;
        if (extra_out) extra_out[i] = extra;
        offsets[i] = run;
        run += n;
    }
    offsets[N] = run;
    return ORC_OK;
}

/* a3: the sample list, pixel index of every slot. */
void orc_sample_list(const int64_t *offsets, int64_t N, int32_t *sample_pixel) {
    for (int64_t i = 0; i < N; ++i)
        for (int64_t t = offsets[i]; t < offsets[i + 1]; ++t) sample_pixel[t] = (int32_t)i;
}

/* ------------------------------------------------------------------------ */
/* a4: renderer stand-in.  The paper path-traces the requested samples with  */
/* Falcor (Sec. 3); here sample k of pixel i is the clean image times a      */
/* unit-mean log-normal factor exp(0.8 Z - 0.32), Z ~ N(0,1) by Box-Muller   */
/* (Box & Muller 1958) from two 24-bit uniforms of SplitMix64 counters:      */
/*   hp = pixel_bits(seed, frame, i),                                        */
/*   b1 = mix(hp + (2k+1) gamma), b2 = mix(hp + (2k+2) gamma),               */
/*   u1 = ((b1 >> 40) + 1/2) 2^-24, u2 = (b2 >> 40) 2^-24,                   */
/*   Z = sqrt(-2 ln u1) cos(2 pi u2).                                        */
/* ------------------------------------------------------------------------ */
double orc_sample_noise(uint64_t seed, uint32_t frame, uint64_t i, uint64_t k) {
    uint64_t hp = orc_pixel_bits(seed, frame, i);
    uint64_t b1 = orc_splitmix64_mix(hp + (2 * k + 1) * ORC_GOLDEN_GAMMA);
    uint64_t b2 = orc_splitmix64_mix(hp + (2 * k + 2) * ORC_GOLDEN_GAMMA);
    double u1 = ((double)(b1 >> 40) + 0.5) * 0x1p-24;
    double u2 = (double)(b2 >> 40) * 0x1p-24;
    double Z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    return exp(0.8 * Z - 0.32);
}

/* rgb: [T][3]; clean: planar [3][N]. */
void orc_render(const double *clean, const int64_t *offsets, int64_t N,
                uint64_t seed, uint32_t frame, double *rgb) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int64_t t = offsets[i]; t < offsets[i + 1]; ++t) {
            double z = orc_sample_noise(seed, frame, (uint64_t)i, (uint64_t)(t - offsets[i]));
            for (int ch = 0; ch < 3; ++ch) rgb[t * 3 + ch] = clean[(int64_t)ch * N + i] * z;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* a5: splat (Eq. stoch_rnoisy) and average-pool pyramid (Eq. app-pyramid). */
/*   L0_i = (sum_{k < floor(s_i)} S_ik + H_i) / s_i,  H_i = w_i S_i,last     */
/*   L^l_xy = 4^-l * sum over the 2^l x 2^l block of L0.                      */
/* layers[l] is planar [3][H>>l][W>>l].                                      */
/* ------------------------------------------------------------------------ */
int orc_splat(const int64_t *offsets, const double *rgb, const double *s, const double *w,
              const int32_t *extra, int W, int H, int L, double *const *layers) {
    if (W < 0 || H < 0 || L < 1) return ORC_ERR_ARG;
    int64_t N = (int64_t)W * H;
    double *L0 = layers[0];
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        int64_t n = offsets[i + 1] - offsets[i];
        int64_t f = n - extra[i];
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.0;
            for (int64_t k = 0; k < f; ++k) acc += rgb[(offsets[i] + k) * 3 + ch];
            if (extra[i]) acc += w[i] * rgb[(offsets[i] + f) * 3 + ch];
            L0[(int64_t)ch * N + i] = acc / s[i];
        }
    }
    for (int l = 1; l < L; ++l) {
        int Wl = W >> l, Hl = H >> l, b = 1 << l;
        int64_t Nl = (int64_t)Wl * Hl;
        double inv = 1.0 / (double)((int64_t)b * b);
        #pragma omp parallel for collapse(2) schedule(static)
        for (int ch = 0; ch < 3; ++ch)
            for (int y = 0; y < Hl; ++y)
                for (int x = 0; x < Wl; ++x) {
                    double acc = 0.0;
                    for (int v = y * b; v < (y + 1) * b; ++v)
                        for (int u = x * b; u < (x + 1) * b; ++u)
                            acc += L0[(int64_t)ch * N + (int64_t)v * W + u];
                    layers[l][(int64_t)ch * Nl + (int64_t)y * Wl + x] = acc * inv;
                }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* a6-a8: gather-pyramid reconstruction (Appendix A).                        */
/* ------------------------------------------------------------------------ */
static int orc_clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* W_t: bilinear sample of prev (planar [3][H][W]) at (x+mv_x, y+mv_y). */
static void orc_warp_at(const double *prev, const float *mv, int W, int H, int x, int y,
                        double out[3]) {
    int64_t N = (int64_t)W * H;
    int64_t idx = (int64_t)y * W + x;
    double X = (double)x + (double)mv[idx];
    double Y = (double)y + (double)mv[N + idx];
    if (X < 0.0) X = 0.0;
    if (X > (double)(W - 1)) X = (double)(W - 1);
    if (Y < 0.0) Y = 0.0;
    if (Y > (double)(H - 1)) Y = (double)(H - 1);
    double x0f = floor(X), y0f = floor(Y);
    double fx = X - x0f, fy = Y - y0f;
    int x0 = (int)x0f, y0 = (int)y0f;
    int x1 = x0 + 1 < W ? x0 + 1 : W - 1;
    int y1 = y0 + 1 < H ? y0 + 1 : H - 1;
    for (int ch = 0; ch < 3; ++ch) {
        const double *P = prev + (int64_t)ch * N;
        double p00 = P[(int64_t)y0 * W + x0], p10 = P[(int64_t)y0 * W + x1];
        double p01 = P[(int64_t)y1 * W + x0], p11 = P[(int64_t)y1 * W + x1];
        out[ch] = (1.0 - fy) * ((1.0 - fx) * p00 + fx * p10) + fy * ((1.0 - fx) * p01 + fx * p11);
    }
}

/* The warped previous frame W_t L_{t-1} over the whole image. */
void orc_warp(const double *prev, const float *mv, int W, int H, double *out) {
    int64_t N = (int64_t)W * H;
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double v[3];
            orc_warp_at(prev, mv, W, H, x, y, v);
            for (int ch = 0; ch < 3; ++ch) out[(int64_t)ch * N + (int64_t)y * W + x] = v[ch];
        }
}

/* One level of Eq. app-recon-coarse / app-recon-mid / app-recon-full.
 *   noisy   : L^l planar [3][Hl][Wl]
 *   logits  : planar [C][Hl][Wl]; C = 25 (coarsest), 29 (with upsampling),
 *             54 (full resolution with temporal kernels)
 *   coarse  : denoised L-hat^{l+1} planar [3][Hl/2][Wl/2], or NULL at the
 *             coarsest level (no upsampling kernel)
 *   warped  : W_t L_{t-1} planar [3][Hl][Wl], or NULL (no temporal term)
 *   mask    : uint8 [Hl][Wl] (nonzero = disoccluded), or NULL
 * The joint softmax spans every kernel present at the pixel (Eq.
 * app-softmax-mid, app-softmax-full); G is Eq. app-gather, U is
 * Eq. app-upsample. */
int orc_reconstruct_level(const double *noisy, const double *logits, int C,
                          const double *coarse, const double *warped, const uint8_t *mask,
                          int Wl, int Hl, double *out) {
    int has_up = coarse != NULL;
    int has_t = warped != NULL;
    int need = 25 + (has_up ? 4 : 0) + (has_t ? 25 : 0);
    if (C < need) return ORC_ERR_ARG;
    int64_t Nl = (int64_t)Wl * Hl;
    int Wc = Wl / 2, Hc = Hl / 2;
    int64_t Nc = (int64_t)Wc * Hc;
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < Hl; ++y)
        for (int x = 0; x < Wl; ++x) {
            int64_t idx = (int64_t)y * Wl + x;
            int use_t = has_t && !(mask && mask[idx]);
            double lg[54];
            int nk = 0;
            for (int k = 0; k < 25; ++k) lg[nk++] = logits[(int64_t)k * Nl + idx];
            if (has_up)
                for (int k = 0; k < 4; ++k) lg[nk++] = logits[(int64_t)(25 + k) * Nl + idx];
            if (use_t)
                for (int k = 0; k < 25; ++k) lg[nk++] = logits[(int64_t)(29 + k) * Nl + idx];
            double m = lg[0];
            for (int k = 1; k < nk; ++k) if (lg[k] > m) m = lg[k];
            double wsum = 0.0;
            double wt[54];
            for (int k = 0; k < nk; ++k) { wt[k] = exp(lg[k] - m); wsum += wt[k]; }
            for (int k = 0; k < nk; ++k) wt[k] /= wsum;
            for (int ch = 0; ch < 3; ++ch) {
                double acc = 0.0;
                /* G(L^l, kappa_d) */
                for (int j = -2; j <= 2; ++j)
                    for (int i = -2; i <= 2; ++i) {
                        int xx = orc_clampi(x + i, 0, Wl - 1), yy = orc_clampi(y + j, 0, Hl - 1);
                        acc += wt[(j + 2) * 5 + (i + 2)] * noisy[(int64_t)ch * Nl + (int64_t)yy * Wl + xx];
                    }
                /* U(L-hat^{l+1}, kappa_u), taps at floor((x+i)/2) */
                if (has_up)
                    for (int j = 0; j <= 1; ++j)
                        for (int i = 0; i <= 1; ++i) {
                            int xc = orc_clampi((x + i) / 2, 0, Wc - 1);
                            int yc = orc_clampi((y + j) / 2, 0, Hc - 1);
                            acc += wt[25 + 2 * j + i] * coarse[(int64_t)ch * Nc + (int64_t)yc * Wc + xc];
                        }
                /* G(W_t L_{t-1}, kappa_t) */
                if (use_t) {
                    int base = has_up ? 29 : 25;
                    for (int j = -2; j <= 2; ++j)
                        for (int i = -2; i <= 2; ++i) {
                            int xx = orc_clampi(x + i, 0, Wl - 1), yy = orc_clampi(y + j, 0, Hl - 1);
                            acc += wt[base + (j + 2) * 5 + (i + 2)] *
                                   warped[(int64_t)ch * Nl + (int64_t)yy * Wl + xx];
                        }
                }
                out[(int64_t)ch * Nl + idx] = acc;
            }
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* a9: tone map (Sec. 5): I = sRGB(tau(alpha (log L (.) beta + k))).         */
/* Reading of the saturation shorthand: per-channel scaling of the natural   */
/* log about the mean of the three log channels; exposure added after, the   */
/* contrast multiplying the sum.  L is floored at 2^-24 before the log.      */
/* ------------------------------------------------------------------------ */
double orc_tau(double x, double s, double h) {
    if (x < s - 1.0) return 0.5 * s * exp((x + 1.0 - s) / s);
    if (x < 1.0 - h) return 0.5 * (1.0 + x);
    return 1.0 - 0.5 * h * exp(-(x + h - 1.0) / h);
}

/* IEC 61966-2-1 sRGB encoding of a linear value in [0,1]. */
double orc_srgb_encode(double v) {
    if (v <= 0.0031308) return 12.92 * v;
    return 1.055 * pow(v, 1.0 / 2.4) - 0.055;
}

void orc_tonemap(const double *hdr, int64_t N, double alpha, double beta, double kexp,
                 double s, double h, double *ldr) {
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double lg[3];
        for (int ch = 0; ch < 3; ++ch) {
            double v = hdr[(int64_t)ch * N + i];
            if (v < 0x1p-24) v = 0x1p-24;
            lg[ch] = log(v);
        }
        double mean = (lg[0] + lg[1] + lg[2]) / 3.0;
        for (int ch = 0; ch < 3; ++ch) {
            double x = alpha * (mean + beta * (lg[ch] - mean) + kexp);
            ldr[(int64_t)ch * N + i] = orc_srgb_encode(orc_tau(x, s, h));
        }
    }
}

/* ======================================================================== */
/* Backward pass (a11).  Each function is the analytic gradient of the      */
/* forward function above it, written out by the chain rule; the pins check */
/* every one against central finite differences of the forward in FP64.    */
/* ======================================================================== */

/* Reconstruction level (App. A): given g = dLoss/d out ([3][Hl][Wl]),
 *   out_c = sum_k w_k v_kc, w = softmax(z over the active kernels)
 *   dLoss/dz_k = w_k (q_k - sum_j w_j q_j), q_k = sum_c g_c v_kc
 *   dLoss/dv_kc = w_k g_c, scattered to the tap's source pixel.
 * grad_logits is overwritten ([C][Hl][Wl], zero for inactive channels);
 * grad_noisy, grad_coarse, grad_warped are accumulated (+=) and may be NULL. */
int orc_reconstruct_level_backward(const double *noisy, const double *logits, int C,
                                   const double *coarse, const double *warped,
                                   const uint8_t *mask, int Wl, int Hl, const double *g,
                                   double *grad_logits, double *grad_noisy,
                                   double *grad_coarse, double *grad_warped) {
    int has_up = coarse != NULL;
    int has_t = warped != NULL;
    int need = 25 + (has_up ? 4 : 0) + (has_t ? 25 : 0);
    if (C < need) return ORC_ERR_ARG;
    int64_t Nl = (int64_t)Wl * Hl;
    int Wc = Wl / 2, Hc = Hl / 2;
    int64_t Nc = (int64_t)Wc * Hc;
    for (int64_t k = 0; k < (int64_t)C * Nl; ++k) grad_logits[k] = 0.0;
    for (int y = 0; y < Hl; ++y)
        for (int x = 0; x < Wl; ++x) {
            int64_t idx = (int64_t)y * Wl + x;
            int use_t = has_t && !(mask && mask[idx]);
            int ch[54];        /* logit channel of each active kernel */
            int64_t src[54];   /* source pixel of each tap */
            int kind[54];      /* 0 noisy, 1 coarse, 2 warped */
            int nk = 0;
            for (int j = -2; j <= 2; ++j)
                for (int i = -2; i <= 2; ++i) {
                    int xx = orc_clampi(x + i, 0, Wl - 1), yy = orc_clampi(y + j, 0, Hl - 1);
                    ch[nk] = (j + 2) * 5 + (i + 2);
                    src[nk] = (int64_t)yy * Wl + xx;
                    kind[nk++] = 0;
                }
            if (has_up)
                for (int j = 0; j <= 1; ++j)
                    for (int i = 0; i <= 1; ++i) {
                        int xc = orc_clampi((x + i) / 2, 0, Wc - 1);
                        int yc = orc_clampi((y + j) / 2, 0, Hc - 1);
                        ch[nk] = 25 + 2 * j + i;
                        src[nk] = (int64_t)yc * Wc + xc;
                        kind[nk++] = 1;
                    }
            if (use_t) {
                int base = has_up ? 29 : 25;
                for (int j = -2; j <= 2; ++j)
                    for (int i = -2; i <= 2; ++i) {
                        int xx = orc_clampi(x + i, 0, Wl - 1), yy = orc_clampi(y + j, 0, Hl - 1);
                        ch[nk] = base + (j + 2) * 5 + (i + 2);
                        src[nk] = (int64_t)yy * Wl + xx;
                        kind[nk++] = 2;
                    }
            }
            double m = logits[(int64_t)ch[0] * Nl + idx];
            for (int k = 1; k < nk; ++k) {
                double v = logits[(int64_t)ch[k] * Nl + idx];
                if (v > m) m = v;
            }
            double wt[54], wsum = 0.0;
            for (int k = 0; k < nk; ++k) {
                wt[k] = exp(logits[(int64_t)ch[k] * Nl + idx] - m);
                wsum += wt[k];
            }
            for (int k = 0; k < nk; ++k) wt[k] /= wsum;
            double q[54], qbar = 0.0;
            for (int k = 0; k < nk; ++k) {
                const double *img = kind[k] == 0 ? noisy : (kind[k] == 1 ? coarse : warped);
                int64_t n = kind[k] == 1 ? Nc : Nl;
                double acc = 0.0;
                for (int c = 0; c < 3; ++c) acc += g[(int64_t)c * Nl + idx] * img[(int64_t)c * n + src[k]];
                q[k] = acc;
                qbar += wt[k] * acc;
            }
            for (int k = 0; k < nk; ++k) {
                grad_logits[(int64_t)ch[k] * Nl + idx] = wt[k] * (q[k] - qbar);
                double *dst = kind[k] == 0 ? grad_noisy : (kind[k] == 1 ? grad_coarse : grad_warped);
                int64_t n = kind[k] == 1 ? Nc : Nl;
                if (dst)
                    for (int c = 0; c < 3; ++c)
                        dst[(int64_t)c * n + src[k]] += wt[k] * g[(int64_t)c * Nl + idx];
            }
        }
    return ORC_OK;
}

/* W_t backward: the bilinear weights of each pixel scatter g to the four
 * previous-frame pixels they read; grad_prev is accumulated. */
void orc_warp_backward(const float *mv, int W, int H, const double *g, double *grad_prev) {
    int64_t N = (int64_t)W * H;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int64_t idx = (int64_t)y * W + x;
            double X = (double)x + (double)mv[idx];
            double Y = (double)y + (double)mv[N + idx];
            if (X < 0.0) X = 0.0;
            if (X > (double)(W - 1)) X = (double)(W - 1);
            if (Y < 0.0) Y = 0.0;
            if (Y > (double)(H - 1)) Y = (double)(H - 1);
            double x0f = floor(X), y0f = floor(Y);
            double fx = X - x0f, fy = Y - y0f;
            int x0 = (int)x0f, y0 = (int)y0f;
            int x1 = x0 + 1 < W ? x0 + 1 : W - 1;
            int y1 = y0 + 1 < H ? y0 + 1 : H - 1;
            for (int c = 0; c < 3; ++c) {
                double gv = g[(int64_t)c * N + idx];
                double *P = grad_prev + (int64_t)c * N;
                P[(int64_t)y0 * W + x0] += (1.0 - fy) * (1.0 - fx) * gv;
                P[(int64_t)y0 * W + x1] += (1.0 - fy) * fx * gv;
                P[(int64_t)y1 * W + x0] += fy * (1.0 - fx) * gv;
                P[(int64_t)y1 * W + x1] += fy * fx * gv;
            }
        }
}

/* Derivative of tau (Sec. 5). */
static double orc_tau_prime(double x, double s, double h) {
    if (x < s - 1.0) return 0.5 * exp((x + 1.0 - s) / s);
    if (x < 1.0 - h) return 0.5;
    return 0.5 * exp(-(x + h - 1.0) / h);
}

/* Derivative of the sRGB encoding. */
static double orc_srgb_prime(double v) {
    if (v <= 0.0031308) return 12.92;
    return 1.055 / 2.4 * pow(v, 1.0 / 2.4 - 1.0);
}

/* Tone-map backward: grad_hdr += d ldr / d hdr applied to grad_ldr. */
void orc_tonemap_backward(const double *hdr, int64_t N, double alpha, double beta, double kexp,
                          double s, double h, const double *grad_ldr, double *grad_hdr) {
    for (int64_t i = 0; i < N; ++i) {
        double lg[3], v[3];
        for (int ch = 0; ch < 3; ++ch) {
            v[ch] = hdr[(int64_t)ch * N + i];
            lg[ch] = log(v[ch] < 0x1p-24 ? 0x1p-24 : v[ch]);
        }
        double mean = (lg[0] + lg[1] + lg[2]) / 3.0;
        double gx[3];
        for (int ch = 0; ch < 3; ++ch) {
            double x = alpha * (mean + beta * (lg[ch] - mean) + kexp);
            double t = orc_tau(x, s, h);
            gx[ch] = grad_ldr[(int64_t)ch * N + i] * orc_srgb_prime(t) * orc_tau_prime(x, s, h);
        }
        double gsum = gx[0] + gx[1] + gx[2];
        for (int j = 0; j < 3; ++j) {
            /* dx_c/dl_j = alpha (beta [c == j] + (1 - beta)/3) */
            double gl = alpha * (beta * gx[j] + (1.0 - beta) / 3.0 * gsum);
            if (v[j] >= 0x1p-24) grad_hdr[(int64_t)j * N + i] += gl / v[j];
        }
    }
}

/* Mean absolute error of the sRGB output against a reference (the spatial
 * loss of Eq. loss_spatial with m = 1); grad = sign(ldr - ref) / n. */
double orc_l1_loss(const double *ldr, const double *ref, int64_t n, double *grad) {
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double d = ldr[i] - ref[i];
        acc += fabs(d);
        if (grad) grad[i] = (d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0)) / (double)n;
    }
    return acc / (double)n;
}

/* Pyramid backward (Eq. app-pyramid): grad_L0 += 4^-l grad_L^l at the
 * coarse pixel each full-resolution pixel pools into. */
void orc_pyramid_backward(double *const *grad_layers, int W, int H, int L, double *grad_L0) {
    int64_t N = (int64_t)W * H;
    for (int l = 1; l < L; ++l) {
        int Wl = W >> l, Hl = H >> l;
        int64_t Nl = (int64_t)Wl * Hl;
        double sc = 1.0 / (double)((int64_t)1 << (2 * l));
        for (int c = 0; c < 3; ++c)
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x)
                    grad_L0[(int64_t)c * N + (int64_t)y * W + x] +=
                        sc * grad_layers[l][(int64_t)c * Nl + (int64_t)(y >> l) * Wl + (x >> l)];
    }
}

/* Splat backward (Eq. stoch_rnoisy with the ramp of Eq. relaxed_holdout):
 *   L0_i = (sum_{k<f} S_ik + w_i S_i,f) / s_i, p_i = s_i - f_i
 *   dL0_i/ds_i = -L0_i / s_i + [extra, linear ramp] h lam (1 - u_i) / p_i^2 S_i,f / s_i
 * (the floor is piecewise constant, so dp/ds = 1 between integers).
 * grad_s is overwritten. */
void orc_splat_backward(const int64_t *offsets, const double *rgb, const double *s,
                        const int32_t *extra, int64_t N, double lambda, int hard, uint64_t seed,
                        uint32_t frame, const double *L0, const double *grad_L0, double *grad_s) {
    double h = (2.0 * lambda) / (2.0 * lambda - 1.0);
    for (int64_t i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int c = 0; c < 3; ++c) acc -= grad_L0[(int64_t)c * N + i] * L0[(int64_t)c * N + i] / s[i];
        if (extra[i] && !hard) {
            double f = floor(s[i]);
            double p = s[i] - f;
            double u = orc_pixel_uniform(seed, frame, (uint64_t)i);
            double r = (lambda / p) * ((u + p) - 1.0);
            if (r > 0.0 && r < 1.0) {
                double dw = h * lambda * (1.0 - u) / (p * p);
                int64_t last = offsets[i + 1] - 1;
                for (int c = 0; c < 3; ++c)
                    acc += grad_L0[(int64_t)c * N + i] * dw * rgb[last * 3 + c] / s[i];
            }
        }
        grad_s[i] = acc;
    }
}

/* Density backward (Sec. 3): s_i = phi B + (1 - phi) B N pi_i with
 * pi = softmax(z) = d / sum d, so
 *   dLoss/dz_j = (1 - phi) B N pi_j (g_j - sum_i pi_i g_i).
 * grad_z is overwritten. */
void orc_density_backward(const double *z, int64_t N, double B, double phi, const double *grad_s,
                          double *grad_z) {
    double m = z[0];
    for (int64_t i = 1; i < N; ++i) if (z[i] > m) m = z[i];
    double S = 0.0;
    for (int64_t i = 0; i < N; ++i) S += exp(z[i] - m);
    double dot = 0.0;
    for (int64_t i = 0; i < N; ++i) dot += exp(z[i] - m) / S * grad_s[i];
    double K = (1.0 - phi) * B * (double)N;
    for (int64_t i = 0; i < N; ++i) {
        double pi = exp(z[i] - m) / S;
        grad_z[i] = K * pi * (grad_s[i] - dot);
    }
}

/* Density forward in FP64 from the sampler logits z (Sec. 3): s_i =
 * phi B + (1 - phi) B N softmax(z)_i.  Used to pin the density backward. */
void orc_density_forward(const double *z, int64_t N, double B, double phi, double *s) {
    double m = z[0];
    for (int64_t i = 1; i < N; ++i) if (z[i] > m) m = z[i];
    double S = 0.0;
    for (int64_t i = 0; i < N; ++i) S += exp(z[i] - m);
    for (int64_t i = 0; i < N; ++i) s[i] = phi * B + (1.0 - phi) * B * (double)N * exp(z[i] - m) / S;
}
