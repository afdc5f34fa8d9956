// a1-a3: budget normalisation, stochastic rounding with the relaxed holdout
// ramp, and the sample list (Sec. 3, Sec. 4.2-4.3 of arXiv 2602.08642).
//
// Two kernels per frame, after one memset of the workspace header:
//   budget_sum_kernel   exact sum of the FP32 density in integer limbs; the
//                       last block rounds it once to FP64 and derives the
//                       budget coefficients a = phi B, c = (1-phi) B N / S.
//   assign_scan_kernel  per pixel: s_i = a + c d_i, n_i, holdout weight; a
//                       single-pass decoupled look-back scan of n_i gives the
//                       offsets; each pixel writes its slots of the sample list.
// Frames of more than 64 tiles of 2048 pixels replace the second kernel by
// two without waits between blocks (assign_tile_kernel: decisions, counts
// and tile sums; offsets_kernel: tile prefix from the earlier tile sums,
// local scan, offsets and sample list), which is faster at full resolution.
//
// Bit-exactness of the count map.  The decisions floor(s_i) and
// u_i > 1 - p_i are those of FP64 round-to-nearest arithmetic.  FP64 is slow
// on this part, so every pixel first evaluates s_i in float-float (error below
// 2^-45 s_i) and decides in FP32 when the decision is further than a safe
// margin from its threshold; only the few pixels within the margin (about
// 2e-6 of them) run the FP64 sequence.
#include <mutex>

#include "spp_internal.cuh"

namespace spp {
namespace {

constexpr int kSumThreads = 256;
constexpr int kLimbs = 11;       // per-thread limb accumulators (32-bit weights)
constexpr int kWords = 13;       // carry-propagated 32-bit words of the total

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kTile = kScanThreads * kScanItems;
// frames of at most this many tiles use the single-pass scan (one launch);
// larger ones the two-pass form without waits between blocks
constexpr int kSinglePassMaxTiles = 64;

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagInc = 2ull << 62;
constexpr int kSpinLimit = 1 << 20;

struct AllocHeader {
    unsigned long long limbs[kLimbs];  // exact sum, limb j has weight 2^(32 j - 149)
    unsigned int blocks_done;          // ticket of the budget sum's last block
    unsigned int tile_counter;         // dynamic tile index of the scan
    int bad_input;
    int valid;                         // 1 when the coefficients below are usable
    double S, a, c, lam, h;
    float a_hi, a_lo, c_hi, c_lo, lam_f, h_f;
    int fast_ok;
};
constexpr size_t kHeaderBytes = 256;
static_assert(sizeof(AllocHeader) <= kHeaderBytes, "alloc header too large");

struct BudgetArgs {
    double budget, phi, lambda;
    int hard;
    int force_exact;
};

// Holdout modes of the assignment (SPP_HOLDOUT_*): 0 ramp, 1 hard, 2 the
// training forward of the Gumbel-softmax estimator, 3 the deterministic
// rounding of DASR (Sec. 4.1).
constexpr int kModeGumbel = 2;
constexpr int kModeDasr = 3;

// ---------------------------------------------------------------- K1
// Every finite FP32 x >= 0 is m 2^(pos - 149) with an integer m < 2^24 and
// pos in [0, 253].  A thread keeps a 128-bit integer sum of m 2^(pos - 32 b)
// for the elements whose 32-bit window pos >> 5 is b or b + 1 (one add with
// carry per element); an element outside that span first moves the sum into
// the thread's 32-bit limbs (limb j weighs 2^(32 j - 149)) and re-bases.
struct ExactAcc {
    unsigned long long lo, hi;
    int b;
};

__device__ __forceinline__ void acc_flush(ExactAcc &A, unsigned long long (&lim)[kLimbs]) {
    if (A.b >= 0) {
        const unsigned long long c0 = A.lo & 0xffffffffull, c1 = A.lo >> 32;
        const unsigned long long c2 = A.hi & 0xffffffffull, c3 = A.hi >> 32;
#pragma unroll
        for (int j = 0; j < kLimbs; ++j) {
            unsigned long long v = 0ull;
            v += (j == A.b) ? c0 : 0ull;
            v += (j == A.b + 1) ? c1 : 0ull;
            v += (j == A.b + 2) ? c2 : 0ull;
            v += (j == A.b + 3) ? c3 : 0ull;
            lim[j] += v;
        }
    }
    A.lo = 0ull;
    A.hi = 0ull;
}

__device__ __forceinline__ void accum_value(float x, ExactAcc &A, unsigned long long (&lim)[kLimbs],
                                            bool &bad) {
    const uint32_t bits = __float_as_uint(x);
    const uint32_t mag = bits & 0x7fffffffu;
    if (mag >= 0x7f800000u || (bits != mag && mag != 0u)) {  // inf, NaN, negative
        bad = true;
        return;
    }
    const uint32_t e = mag >> 23;
    const unsigned long long m = (mag & 0x7fffffu) | (e ? 0x800000u : 0u);
    const int pos = e ? static_cast<int>(e) - 1 : 0;  // x = m 2^(pos - 149)
    const int w = pos >> 5;
    if (w < A.b || w > A.b + 1) {  // rare for data spanning < 2^32 in range
        acc_flush(A, lim);
        A.b = w > 0 ? w - 1 : 0;
    }
    const int sh = pos - 32 * A.b;  // 0 .. 63
    const unsigned long long vlo = m << sh;
    const unsigned long long vhi = sh > 40 ? (m >> (64 - sh)) : 0ull;
    A.lo += vlo;
    A.hi += vhi + (A.lo < vlo ? 1ull : 0ull);
}

// Correctly rounded FP64 value of the exact total (single thread): carry the
// limbs into 32-bit words, take the 64 bits below the leading one, round to
// nearest even with the remaining bits as sticky.
__device__ double round_limbs(const unsigned long long *limbs) {
    uint32_t w[kWords];
    unsigned long long carry = 0ull;
#pragma unroll
    for (int j = 0; j < kLimbs; ++j) {
        const unsigned long long v = limbs[j] + carry;
        w[j] = static_cast<uint32_t>(v & 0xffffffffull);
        carry = v >> 32;
    }
    w[kLimbs] = static_cast<uint32_t>(carry & 0xffffffffull);
    w[kLimbs + 1] = static_cast<uint32_t>(carry >> 32);
    int t = -1;
#pragma unroll
    for (int j = 0; j < kWords; ++j)
        if (w[j]) t = j;
    if (t < 0) return 0.0;
    if (t <= 1) {  // below 2^64 units of 2^-149: convert in two exact steps
        const unsigned long long x =
            static_cast<unsigned long long>(w[0]) | (static_cast<unsigned long long>(w[1]) << 32);
        if ((x >> 53) == 0ull) return __dmul_rn(__ull2double_rn(x), 0x1p-149);
    }
    uint32_t w1 = 0u, w2 = 0u, below = 0u;
#pragma unroll
    for (int j = 0; j < kWords; ++j) {
        if (j == t - 1) w1 = w[j];
        if (j == t - 2) w2 = w[j];
        if (j < t - 2) below |= w[j];
    }
    const int lz = __clz(w[t]);
    unsigned long long a = (static_cast<unsigned long long>(w[t]) << 32) | w1;
    uint32_t b = w2;
    if (lz > 0) {
        a = (a << lz) | static_cast<unsigned long long>(b >> (32 - lz));
        b = b << lz;
    }
    // a holds the leading 64 bits (bit 63 set); value = a 2^(P - 63 - 149)
    const int P = 32 * t + 31 - lz;
    unsigned long long mant = a >> 11;
    const unsigned long long rbit = (a >> 10) & 1ull;
    const bool sticky = (a & 0x3ffull) != 0ull || b != 0u || below != 0u;
    int exp2 = P - 149;  // value = mant 2^(exp2 - 52)
    if (rbit && (sticky || (mant & 1ull))) {
        ++mant;
        if (mant == (1ull << 53)) {
            mant >>= 1;
            ++exp2;
        }
    }
    const unsigned long long bits = (static_cast<unsigned long long>(exp2 + 1023) << 52) |
                                    (mant & ((1ull << 52) - 1ull));
    return __longlong_as_double(static_cast<long long>(bits));
}

__device__ void finalize_budget(AllocHeader *hdr, const unsigned long long *limbs, int bad,
                                long long N, const BudgetArgs &args, int32_t *status) {
    const double S = round_limbs(limbs);
    hdr->S = S;
    if (bad || !(S > 0.0)) {
        set_status(status, SPP_ERR_INPUT);
        hdr->valid = 0;
        return;
    }
    // The FP64 round-to-nearest sequence of Sec. 3 (no contraction).
    const double a = __dmul_rn(args.phi, args.budget);
    const double k = __dmul_rn(__dsub_rn(1.0, args.phi), args.budget);
    const double num = __dmul_rn(k, static_cast<double>(N));
    const double c = __ddiv_rn(num, S);
    const double two_lam = __dmul_rn(2.0, args.lambda);
    const double h = __ddiv_rn(two_lam, __dsub_rn(two_lam, 1.0));
    hdr->a = a;
    hdr->c = c;
    hdr->lam = args.lambda;
    hdr->h = h;
    const float c_hi = __double2float_rn(c);
    const float a_hi = __double2float_rn(a);
    hdr->c_hi = c_hi;
    hdr->c_lo = __double2float_rn(__dsub_rn(c, static_cast<double>(c_hi)));
    hdr->a_hi = a_hi;
    hdr->a_lo = __double2float_rn(__dsub_rn(a, static_cast<double>(a_hi)));
    hdr->lam_f = __double2float_rn(args.lambda);
    hdr->h_f = __double2float_rn(h);
    const bool c_ok = c >= 0x1p-60 && c <= 0x1p60;
    const bool a_ok = a == 0.0 || (a >= 0x1p-60 && a <= 0x1p60);
    hdr->fast_ok = (c_ok && a_ok && !args.force_exact) ? 1 : 0;
    __threadfence();
    hdr->valid = 1;
}

template <int U>
__global__ void __launch_bounds__(kSumThreads)
budget_sum_kernel(const float *__restrict__ d, long long N, AllocHeader *hdr, BudgetArgs args,
                  int32_t *status) {
    pdl_wait();
    pdl_trigger();
    unsigned long long lim[kLimbs];
#pragma unroll
    for (int j = 0; j < kLimbs; ++j) lim[j] = 0ull;
    ExactAcc A;
    A.lo = 0ull;
    A.hi = 0ull;
    A.b = -100;
    bool bad = false;
    const long long nthreads = static_cast<long long>(gridDim.x) * blockDim.x;
    const long long gtid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    const long long n4 = N >> 2;
    const float4 *d4 = reinterpret_cast<const float4 *>(d);
    // U independent vector loads in flight per thread and iteration.  Chunk
    // sums: when the 4U values of a thread are finite, non-negative, normal
    // (or zero) and their exponents span at most 32 binades, the integer
    //   S = sum of m_i 2^(e_i - e_min)  (m_i the 24-bit significand)
    // is exact in 64 bits (below 4U 2^56), and the chunk is S 2^(e_min - 150),
    // i.e. S at bit position e_min - 1 of the accumulator: one shift-and-add
    // of 128 bits per chunk instead of one per value.  Other chunks (and the
    // tail) take the per-value path.  After at most 32 chunk adds the 128-bit
    // sum moves into the limbs, so it cannot overflow (each chunk add is below
    // 2^122, each per-value add below 2^87).
    int nadd = 0;
    for (long long q0 = gtid; q0 < n4; q0 += U * nthreads) {
        float4 v4[U];
#pragma unroll
        for (int r = 0; r < U; ++r) {
            const long long q = q0 + r * nthreads;
            v4[r] = q < n4 ? __ldg(d4 + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const float *v = reinterpret_cast<const float *>(v4);
        uint32_t emin = 255u, emax = 0u;
        bool ok = true;
#pragma unroll
        for (int r = 0; r < 4 * U; ++r) {
            const uint32_t bits = __float_as_uint(v[r]);
            const uint32_t e = bits >> 23;  // the sign bit makes e > 255
            // finite, non-negative, and normal or +0
            ok &= e < 255u && (e != 0u || bits == 0u);
            emin = min(emin, bits ? e : 255u);
            emax = max(emax, bits ? e : 0u);
        }
        if (ok && (emax < emin || emax - emin <= 32u)) {
            if (emax >= emin) {  // not all zero
                unsigned long long S = 0ull;
#pragma unroll
                for (int r = 0; r < 4 * U; ++r) {
                    const uint32_t bits = __float_as_uint(v[r]);
                    const uint32_t m = bits ? ((bits & 0x7fffffu) | 0x800000u) : 0u;
                    const uint32_t sh = (bits >> 23) - emin;  // 0 .. 32 when m != 0
                    const uint32_t lo = __funnelshift_lc(0u, m, sh);
                    const uint32_t hi = __funnelshift_lc(m, 0u, sh);
                    S += (static_cast<unsigned long long>(hi) << 32) | lo;
                }
                const int pos = static_cast<int>(emin) - 1;  // S 2^(pos - 149)
                const bool empty = A.lo == 0ull && A.hi == 0ull;
                if (!empty && (pos < 32 * A.b || pos - 32 * A.b > 63 || nadd >= 32)) {
                    acc_flush(A, lim);
                    nadd = 0;
                }
                if (A.lo == 0ull && A.hi == 0ull) A.b = pos >> 5;
                const int sh = pos - 32 * A.b;  // 0 .. 63
                const unsigned long long add_lo = S << sh;
                const unsigned long long add_hi = sh ? (S >> (64 - sh)) : 0ull;
                A.lo += add_lo;
                A.hi += add_hi + (A.lo < add_lo ? 1ull : 0ull);
                ++nadd;
            }
        } else {
#pragma unroll
            for (int r = 0; r < 4 * U; ++r) accum_value(v[r], A, lim, bad);
        }
    }
    for (long long i = (n4 << 2) + gtid; i < N; i += nthreads) accum_value(d[i], A, lim, bad);
    acc_flush(A, lim);

    __shared__ unsigned long long s_part[kSumThreads / 32][kLimbs];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kLimbs; ++j) {
        unsigned long long v = lim[j];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) s_part[warp][j] = v;
    }
    const int any_bad = __syncthreads_or(bad ? 1 : 0);
    if (threadIdx.x < kLimbs) {
        unsigned long long v = 0ull;
        for (int w = 0; w < kSumThreads / 32; ++w) v += s_part[w][threadIdx.x];
        if (v) atomicAdd(&hdr->limbs[threadIdx.x], v);
    }
    if (threadIdx.x == 0 && any_bad) atomicOr(&hdr->bad_input, 1);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int t = atomicAdd(&hdr->blocks_done, 1u);
        s_last = (t == gridDim.x - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
        // the last block gathers the limbs in parallel, then one thread rounds
        __shared__ unsigned long long s_limbs[kLimbs];
        __shared__ int s_bad;
        __threadfence();
        if (threadIdx.x < kLimbs)
            s_limbs[threadIdx.x] = *reinterpret_cast<volatile unsigned long long *>(&hdr->limbs[threadIdx.x]);
        if (threadIdx.x == kLimbs) s_bad = *reinterpret_cast<volatile int *>(&hdr->bad_input);
        __syncthreads();
        if (threadIdx.x == 0) finalize_budget(hdr, s_limbs, s_bad, N, args, status);
    }
}

// ---------------------------------------------------------------- K2
struct Coef {
    double a, c, lam, h;
    float a_hi, a_lo, c_hi, c_lo, lam_f, h_f;
    int hard, fast;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

struct PixelOut {
    int n;
    float w, s;
};

// FP64 sequence, operation for operation the definition of Sec. 3 and 4.2-4.3.
// Returned by value so that the caller's per-item arrays stay in registers.
__device__ __noinline__ PixelOut assign_exact(float d, uint64_t bits, double ka, double kc,
                                              double klam, double kh, int hard) {
    const double u = __dmul_rn(__ull2double_rn(bits >> 16), 0x1p-48);
    const double m = __dmul_rn(kc, static_cast<double>(d));
    const double sd = __dadd_rn(ka, m);
    const double f = floor(sd);
    const double p = __dsub_rn(sd, f);
    const double t = __dsub_rn(1.0, p);
    if (hard == kModeDasr) {
        // Eq. kuz_fw: round(s) samples, halves up (p is exact); the splat
        // divides by max(n, 1), which s_out carries in this mode
        PixelOut r;
        r.n = static_cast<int>(f) + (p >= 0.5 ? 1 : 0);
        r.w = 1.0f;
        r.s = static_cast<float>(r.n > 1 ? r.n : 1);
        return r;
    }
    if (hard == kModeGumbel) {
        // binary concrete relaxation: the extra sample is always traced,
        // weighted by sigma(lambda (ln(p / (1 - p)) + ln(u / (1 - u))))
        PixelOut r;
        const bool extra = p > 0.0;
        double wd = 1.0;
        if (extra) {
            const double x = __dmul_rn(klam, __dadd_rn(log(__ddiv_rn(p, t)),
                                                       log(__ddiv_rn(u, __dsub_rn(1.0, u)))));
            wd = __ddiv_rn(1.0, __dadd_rn(1.0, exp(-x)));
        }
        r.n = static_cast<int>(f) + (extra ? 1 : 0);
        r.w = __double2float_rn(wd);
        r.s = __double2float_rn(sd);
        return r;
    }
    const bool extra = (p > 0.0) && (u > t);
    double wd = 1.0;
    if (extra && !hard) {
        const double q = __ddiv_rn(klam, p);
        const double v = __dsub_rn(__dadd_rn(u, p), 1.0);
        double r = __dmul_rn(q, v);
        r = r < 0.0 ? 0.0 : (r > 1.0 ? 1.0 : r);
        wd = __dmul_rn(kh, r);
    }
    PixelOut r;
    r.n = static_cast<int>(f) + (extra ? 1 : 0);
    r.w = __double2float_rn(wd);
    r.s = __double2float_rn(sd);
    return r;
}

// Float-float filter.  Returns false when a decision is within the margin of
// its threshold (the caller then runs assign_exact).
__device__ __forceinline__ bool assign_fast(float d, uint64_t bits, const Coef &k, int &n,
                                            float &w, float &s) {
    // s = a + c d in float-float
    const float ph = __fmul_rn(k.c_hi, d);
    float pl = __fmaf_rn(k.c_hi, d, -ph);
    pl = __fmaf_rn(k.c_lo, d, pl);
    float s1, e1;
    two_sum(k.a_hi, ph, s1, e1);
    const float e = __fadd_rn(e1, __fadd_rn(k.a_lo, pl));
    const float sh = __fadd_rn(s1, e);
    const float sl = __fsub_rn(e, __fsub_rn(sh, s1));
    if (!(sh < 4194304.0f)) return false;
    const float E = __fmaf_rn(sh, 0x1p-40f, 0x1p-90f);  // bound on |s_ff - s_fp64|
    float f = floorf(sh);
    if (sh == f && sl < 0.0f) f = __fsub_rn(f, 1.0f);
    const float p1 = __fsub_rn(sh, f);  // exact
    const float plow = __fadd_rn(p1, sl);  // p, distance to floor
    float hh, he;
    two_sum(1.0f, -p1, hh, he);
    const float hl = __fsub_rn(he, sl);  // 1 - p = hh + hl
    if (plow < 2.0f * E || __fadd_rn(hh, hl) < 2.0f * E) return false;
    const float uh = __fmul_rn(static_cast<float>(static_cast<uint32_t>(bits >> 40)), 0x1p-24f);
    const float ul = __fmul_rn(static_cast<float>(static_cast<uint32_t>((bits >> 16) & 0xffffffull)),
                               0x1p-48f);
    float vh, ve;
    two_sum(uh, -hh, vh, ve);
    const float v = __fadd_rn(vh, __fadd_rn(ve, __fsub_rn(ul, hl)));  // u + p - 1
    const float thr = fmaxf(0x1p-20f, 4.0f * E);
    if (fabsf(v) < thr) return false;
    const bool extra = v > 0.0f;
    float wf = 1.0f;
    if (extra && !k.hard) {
        float r = __fmul_rn(__fdividef(k.lam_f, plow), v);  // 2-ulp quotient suffices for w
        r = fminf(fmaxf(r, 0.0f), 1.0f);
        wf = __fmul_rn(k.h_f, r);
    }
    n = static_cast<int>(f) + (extra ? 1 : 0);
    w = wf;
    s = sh;
    return true;
}

__device__ __forceinline__ unsigned long long ld_state(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

__device__ __forceinline__ void st_state(unsigned long long *p, unsigned long long v) {
    atomicExch(p, v);
}

// Source of the uniforms u_i: the counter-based white noise (mask == null),
// or a tiled T x T blue-noise rank mask (Sec. 6.3):
//   u48 = (rank[y mod T][x mod T] 2^(48 - 2 log2 T) + 2^(47 - 2 log2 T) + off48) mod 2^48
// with off48 = t G48 + (mix(seed) >> 16) mod 2^48 set by the host.
struct Dither {
    const uint16_t *mask = nullptr;
    int W = 0, log2T = 0;
    uint64_t off48 = 0;
};

__device__ __forceinline__ uint64_t dither_bits(const Dither &dt, long long i) {
    const int y = static_cast<int>(i / dt.W), x = static_cast<int>(i - static_cast<long long>(y) * dt.W);
    const int T = 1 << dt.log2T;
    const uint64_t r = __ldg(dt.mask + ((y & (T - 1)) << dt.log2T) + (x & (T - 1)));
    const uint64_t u48 = ((r << (48 - 2 * dt.log2T)) + (1ull << (47 - 2 * dt.log2T)) + dt.off48) &
                         0xFFFFFFFFFFFFull;
    return u48 << 16;
}

__global__ void __launch_bounds__(kScanThreads, 4)
assign_scan_kernel(const float *__restrict__ d, long long N, const AllocHeader *hdr_c,
                   AllocHeader *hdr, unsigned long long *tile_state, uint64_t key, Dither dither,
                   int hard, int stall_tile1,
                   int32_t *__restrict__ counts, int32_t *__restrict__ offsets,
                   int32_t *__restrict__ sample_pixel, long long capacity, float *__restrict__ s_out,
                   float *__restrict__ w_out, long long *total, int32_t *status, int num_tiles) {
    __shared__ int s_tile;
    __shared__ int s_warp_excl[kScanThreads / 32];
    __shared__ int s_warp_tot[kScanThreads / 32];
    __shared__ int s_prefix;
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x == 0) s_tile = static_cast<int>(atomicAdd(&hdr->tile_counter, 1u));
    __syncthreads();
    const int tile = s_tile;
    const long long base = static_cast<long long>(tile) * kTile +
                           static_cast<long long>(threadIdx.x) * kScanItems;

    Coef k;
    const int valid = hdr_c->valid;
    k.a = hdr_c->a;
    k.c = hdr_c->c;
    k.lam = hdr_c->lam;
    k.h = hdr_c->h;
    k.a_hi = hdr_c->a_hi;
    k.a_lo = hdr_c->a_lo;
    k.c_hi = hdr_c->c_hi;
    k.c_lo = hdr_c->c_lo;
    k.lam_f = hdr_c->lam_f;
    k.h_f = hdr_c->h_f;
    k.hard = hard;
    k.fast = hdr_c->fast_ok;

    float dv[kScanItems];
    const bool full = base + kScanItems <= N;
    if (full) {
        const float4 v0 = __ldcs(reinterpret_cast<const float4 *>(d + base));
        const float4 v1 = __ldcs(reinterpret_cast<const float4 *>(d + base) + 1);
        dv[0] = v0.x; dv[1] = v0.y; dv[2] = v0.z; dv[3] = v0.w;
        dv[4] = v1.x; dv[5] = v1.y; dv[6] = v1.z; dv[7] = v1.w;
    } else {
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) dv[q] = (base + q < N) ? d[base + q] : 0.0f;
    }
    int n[kScanItems];
    float wv[kScanItems], sv[kScanItems];
    int tsum = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        const long long i = base + q;
        n[q] = 0;
        wv[q] = 1.0f;
        sv[q] = 1.0f;
        if (i < N && valid) {
            const uint64_t bits = dither.mask ? dither_bits(dither, i)
                                              : stream_bits(key, static_cast<uint64_t>(i));
            int nq = 0;
            float wq = 1.0f, sq = 1.0f;
            bool done = false;
            if (k.fast) done = assign_fast(dv[q], bits, k, nq, wq, sq);
            if (!done) {
                const PixelOut r = assign_exact(dv[q], bits, k.a, k.c, k.lam, k.h, k.hard);
                nq = r.n;
                wq = r.w;
                sq = r.s;
            }
            n[q] = nq;
            wv[q] = wq;
            sv[q] = sq;
        }
        tsum += n[q];
    }

    // block-wide exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = tsum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) s_warp_tot[warp] = incl;
    __syncthreads();
    __shared__ int s_agg;
    __shared__ int s_first[kScanThreads / 32];
    __shared__ int s_part[kScanThreads / 32];
    if (warp == 0) {
        const int wt = lane < kScanThreads / 32 ? s_warp_tot[lane] : 0;
        int wincl = wt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wincl, off);
            if (lane >= off) wincl += y;
        }
        if (lane < kScanThreads / 32) s_warp_excl[lane] = wincl - wt;
        const int agg = __shfl_sync(0xffffffffu, wincl, kScanThreads / 32 - 1);
        if (lane == 0) {
            s_agg = agg;
            if (!(stall_tile1 && tile == 1))  // the test of the bounded waits publishes nothing
                st_state(&tile_state[tile], (tile == 0 ? kFlagInc : kFlagAgg) |
                                                static_cast<unsigned int>(agg));
        }
    }
    __syncthreads();
    // decoupled look-back with the whole block: each round reads the states of
    // the 256 nearest predecessors not yet accounted for and stops at the
    // nearest one that already holds an inclusive prefix
    long long excl = 0;
    if (tile > 0) {
        int j = tile - 1;
        while (true) {
            const int idx = j - static_cast<int>(threadIdx.x);
            unsigned long long st = kFlagInc;  // before tile 0: an empty inclusive prefix
            if (idx >= 0) {
                st = ld_state(&tile_state[idx]);
                int spins = 0;
                while ((st >> 62) == 0ull) {
                    if (++spins > kSpinLimit) {
                        set_status(status, SPP_ERR_TIMEOUT);
                        st = kFlagInc;
                        break;
                    }
                    __nanosleep(64);
                    st = ld_state(&tile_state[idx]);
                }
            }
            const unsigned inc = __ballot_sync(0xffffffffu, (st >> 62) == 2ull);
            if (lane == 0) s_first[warp] = inc ? warp * 32 + __ffs(inc) - 1 : 0x7fffffff;
            __syncthreads();
            int first = 0x7fffffff;
#pragma unroll
            for (int w = 0; w < kScanThreads / 32; ++w) first = min(first, s_first[w]);
            int val = static_cast<int>(threadIdx.x) <= first ? static_cast<int>(st & 0xffffffffull) : 0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) val += __shfl_down_sync(0xffffffffu, val, off);
            if (lane == 0) s_part[warp] = val;
            __syncthreads();
#pragma unroll
            for (int w = 0; w < kScanThreads / 32; ++w) excl += s_part[w];
            __syncthreads();  // s_first / s_part are reused by the next round
            if (first != 0x7fffffff) break;
            j -= kScanThreads;
        }
        if (threadIdx.x == 0 && !(stall_tile1 && tile == 1))
            st_state(&tile_state[tile],
                     kFlagInc | static_cast<unsigned int>(excl + static_cast<long long>(s_agg)));
    }
    if (threadIdx.x == 0) s_prefix = static_cast<int>(excl);
    __syncthreads();

    int run = s_prefix + s_warp_excl[warp] + (incl - tsum);
    int off[kScanItems];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        off[q] = run;
        run += n[q];
    }
    if (full) {
        int4 *o4 = reinterpret_cast<int4 *>(offsets + base);
        o4[0] = make_int4(off[0], off[1], off[2], off[3]);
        o4[1] = make_int4(off[4], off[5], off[6], off[7]);
        float4 *s4 = reinterpret_cast<float4 *>(s_out + base);
        s4[0] = make_float4(sv[0], sv[1], sv[2], sv[3]);
        s4[1] = make_float4(sv[4], sv[5], sv[6], sv[7]);
        float4 *w4 = reinterpret_cast<float4 *>(w_out + base);
        w4[0] = make_float4(wv[0], wv[1], wv[2], wv[3]);
        w4[1] = make_float4(wv[4], wv[5], wv[6], wv[7]);
        if (counts) {
            int4 *c4 = reinterpret_cast<int4 *>(counts + base);
            c4[0] = make_int4(n[0], n[1], n[2], n[3]);
            c4[1] = make_int4(n[4], n[5], n[6], n[7]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            if (base + q < N) {
                offsets[base + q] = off[q];
                s_out[base + q] = sv[q];
                w_out[base + q] = wv[q];
                if (counts) counts[base + q] = n[q];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        for (int r = 0; r < n[q]; ++r) {
            const long long t = static_cast<long long>(off[q]) + r;
            if (t < capacity) sample_pixel[t] = static_cast<int32_t>(base + q);
        }
    }
    // the owner of the last pixel closes the scan
    if (base <= N - 1 && N - 1 < base + kScanItems) {
        offsets[N] = run;
        *total = run;
        if (static_cast<long long>(run) > capacity) set_status(status, SPP_ERR_CAPACITY);
    }
    (void)num_tiles;
}

// ------------------------------------------- two-pass form (large frames)
// The same sample map without waits between blocks: assign_tile_kernel
// decides every pixel (counts, s, holdout weight) and the sum of its tile;
// offsets_kernel takes its tile's prefix as the sum of the earlier tiles'
// sums, scans its pixels and writes the offsets and the sample list.  Used
// when the frame has many tiles (the counts are an output anyway, so the
// second pass re-reads them from L2); small frames keep the single pass.
__global__ void __launch_bounds__(kScanThreads, 4)
assign_tile_kernel(const float *__restrict__ d, long long N, const AllocHeader *hdr_c,
                   uint64_t key, Dither dither, int hard, int32_t *__restrict__ counts,
                   float *__restrict__ s_out, float *__restrict__ w_out,
                   int *__restrict__ tile_sums) {
    pdl_wait();
    pdl_trigger();
    const int tile = blockIdx.x;
    const long long base = static_cast<long long>(tile) * kTile +
                           static_cast<long long>(threadIdx.x) * kScanItems;
    Coef k;
    const int valid = hdr_c->valid;
    k.a = hdr_c->a;
    k.c = hdr_c->c;
    k.lam = hdr_c->lam;
    k.h = hdr_c->h;
    k.a_hi = hdr_c->a_hi;
    k.a_lo = hdr_c->a_lo;
    k.c_hi = hdr_c->c_hi;
    k.c_lo = hdr_c->c_lo;
    k.lam_f = hdr_c->lam_f;
    k.h_f = hdr_c->h_f;
    k.hard = hard;
    k.fast = hdr_c->fast_ok;

    float dv[kScanItems];
    const bool full = base + kScanItems <= N;
    if (full) {
        const float4 v0 = __ldcs(reinterpret_cast<const float4 *>(d + base));
        const float4 v1 = __ldcs(reinterpret_cast<const float4 *>(d + base) + 1);
        dv[0] = v0.x; dv[1] = v0.y; dv[2] = v0.z; dv[3] = v0.w;
        dv[4] = v1.x; dv[5] = v1.y; dv[6] = v1.z; dv[7] = v1.w;
    } else {
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) dv[q] = (base + q < N) ? d[base + q] : 0.0f;
    }
    int n[kScanItems];
    float wv[kScanItems], sv[kScanItems];
    int tsum = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        const long long i = base + q;
        n[q] = 0;
        wv[q] = 1.0f;
        sv[q] = 1.0f;
        if (i < N && valid) {
            const uint64_t bits = dither.mask ? dither_bits(dither, i)
                                              : stream_bits(key, static_cast<uint64_t>(i));
            int nq = 0;
            float wq = 1.0f, sq = 1.0f;
            bool done = false;
            if (k.fast) done = assign_fast(dv[q], bits, k, nq, wq, sq);
            if (!done) {
                const PixelOut r = assign_exact(dv[q], bits, k.a, k.c, k.lam, k.h, k.hard);
                nq = r.n;
                wq = r.w;
                sq = r.s;
            }
            n[q] = nq;
            wv[q] = wq;
            sv[q] = sq;
        }
        tsum += n[q];
    }
    if (full) {
        int4 *c4 = reinterpret_cast<int4 *>(counts + base);
        c4[0] = make_int4(n[0], n[1], n[2], n[3]);
        c4[1] = make_int4(n[4], n[5], n[6], n[7]);
        float4 *s4 = reinterpret_cast<float4 *>(s_out + base);
        s4[0] = make_float4(sv[0], sv[1], sv[2], sv[3]);
        s4[1] = make_float4(sv[4], sv[5], sv[6], sv[7]);
        float4 *w4 = reinterpret_cast<float4 *>(w_out + base);
        w4[0] = make_float4(wv[0], wv[1], wv[2], wv[3]);
        w4[1] = make_float4(wv[4], wv[5], wv[6], wv[7]);
    } else {
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            if (base + q < N) {
                counts[base + q] = n[q];
                s_out[base + q] = sv[q];
                w_out[base + q] = wv[q];
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) tsum += __shfl_down_sync(0xffffffffu, tsum, off);
    __shared__ int s_w[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = tsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
#pragma unroll
        for (int w = 0; w < kScanThreads / 32; ++w) t += s_w[w];
        tile_sums[tile] = t;
    }
}

__global__ void __launch_bounds__(kScanThreads)
offsets_kernel(const int32_t *__restrict__ counts, long long N, const int *__restrict__ tile_sums,
               int num_tiles, int32_t *__restrict__ offsets, int32_t *__restrict__ sample_pixel,
               long long capacity, long long *total, int32_t *status) {
    pdl_wait();
    pdl_trigger();
    const int tile = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ int s_w[kScanThreads / 32];
    __shared__ int s_pre;
    // this tile's prefix: the sum of the earlier tiles' sums
    int pre = 0;
    for (int t = threadIdx.x; t < tile; t += kScanThreads) pre += tile_sums[t];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) pre += __shfl_down_sync(0xffffffffu, pre, off);
    if (lane == 0) s_w[warp] = pre;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
#pragma unroll
        for (int w = 0; w < kScanThreads / 32; ++w) t += s_w[w];
        s_pre = t;
    }
    __syncthreads();
    const long long base = static_cast<long long>(tile) * kTile +
                           static_cast<long long>(threadIdx.x) * kScanItems;
    int n[kScanItems];
    const bool full = base + kScanItems <= N;
    if (full) {
        const int4 c0 = reinterpret_cast<const int4 *>(counts + base)[0];
        const int4 c1 = reinterpret_cast<const int4 *>(counts + base)[1];
        n[0] = c0.x; n[1] = c0.y; n[2] = c0.z; n[3] = c0.w;
        n[4] = c1.x; n[5] = c1.y; n[6] = c1.z; n[7] = c1.w;
    } else {
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) n[q] = base + q < N ? counts[base + q] : 0;
    }
    int tsum = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) tsum += n[q];
    int incl = tsum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    __syncthreads();  // s_w is reused
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    int before = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w)
        if (w < warp) before += s_w[w];
    int run = s_pre + before + incl - tsum;
    int off[kScanItems];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        off[q] = run;
        run += n[q];
    }
    if (full) {
        int4 *o4 = reinterpret_cast<int4 *>(offsets + base);
        o4[0] = make_int4(off[0], off[1], off[2], off[3]);
        o4[1] = make_int4(off[4], off[5], off[6], off[7]);
    } else {
#pragma unroll
        for (int q = 0; q < kScanItems; ++q)
            if (base + q < N) offsets[base + q] = off[q];
    }
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        for (int r = 0; r < n[q]; ++r) {
            const long long t = static_cast<long long>(off[q]) + r;
            if (t < capacity) sample_pixel[t] = static_cast<int32_t>(base + q);
        }
    }
    // the owner of the last pixel closes the scan
    if (base <= N - 1 && N - 1 < base + kScanItems) {
        offsets[N] = run;
        *total = run;
        if (static_cast<long long>(run) > capacity) set_status(status, SPP_ERR_CAPACITY);
    }
    (void)num_tiles;
}

// ------------------------------------------------- systematic rounding
// The exact-integer-total variant: pixel intervals of length s_i laid end to
// end from a frame offset U, in 32.32 fixed point (q_i = s_i 2^32 rounded to
// nearest even, an exact integer prefix P):
//   offsets_i = (P_{i-1} + U) >> 32, n_i = offsets_{i+1} - offsets_i,
//   extra_i iff a_i + p_i >= 2^32 with a_i = (P_{i-1} + U) mod 2^32 and
//   p_i = q_i mod 2^32; the holdout ramp of Sec. 4.3 at u = a_i 2^-32.
// Reduce-then-scan with no waits between blocks: tile sums of q, one block
// scans them, then every tile scans its own pixels from its prefix.
__device__ __forceinline__ long long fixed_q(float d, double a, double c) {
    const double sd = __dadd_rn(a, __dmul_rn(c, static_cast<double>(d)));
    return __double2ll_rn(__dmul_rn(sd, 4294967296.0));
}

__device__ __forceinline__ long long block_excl_scan_ll(long long v, long long &total) {
    __shared__ long long s_w[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    long long before = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        const long long t = s_w[w];
        if (w < warp) before += t;
        all += t;
    }
    __syncthreads();  // s_w may be reused by the caller's next scan
    total = all;
    return before + incl - v;
}

__global__ void __launch_bounds__(kScanThreads)
sys_tile_sum_kernel(const float *__restrict__ d, long long N, const AllocHeader *hdr,
                    long long *__restrict__ tile_sums) {
    const long long base = static_cast<long long>(blockIdx.x) * kTile +
                           static_cast<long long>(threadIdx.x) * kScanItems;
    const int valid = hdr->valid;
    const double a = hdr->a, c = hdr->c;
    long long sum = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < N && valid) sum += fixed_q(d[base + q], a, c);
    long long total;
    (void)block_excl_scan_ll(sum, total);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Exclusive scan of the tile sums in place, one block.
__global__ void __launch_bounds__(kScanThreads)
sys_scan_tiles_kernel(long long *__restrict__ tile_sums, int num_tiles) {
    const int per = (num_tiles + kScanThreads - 1) / kScanThreads;
    const int t0 = static_cast<int>(threadIdx.x) * per;
    long long mine = 0;
    for (int k = 0; k < per && t0 + k < num_tiles; ++k) mine += tile_sums[t0 + k];
    long long total;
    long long run = block_excl_scan_ll(mine, total);
    for (int k = 0; k < per && t0 + k < num_tiles; ++k) {
        const long long v = tile_sums[t0 + k];
        tile_sums[t0 + k] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(kScanThreads)
sys_assign_kernel(const float *__restrict__ d, long long N, const AllocHeader *hdr,
                  const long long *__restrict__ tile_prefix, unsigned long long U, int hard,
                  int32_t *__restrict__ counts, int32_t *__restrict__ offsets,
                  int32_t *__restrict__ sample_pixel, long long capacity,
                  float *__restrict__ s_out, float *__restrict__ w_out, long long *total,
                  int32_t *status) {
    const long long base = static_cast<long long>(blockIdx.x) * kTile +
                           static_cast<long long>(threadIdx.x) * kScanItems;
    const int valid = hdr->valid;
    const double a = hdr->a, c = hdr->c, lam = hdr->lam, h = hdr->h;
    long long qv[kScanItems];
    long long sum = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        qv[q] = (base + q < N && valid) ? fixed_q(d[base + q], a, c) : 0;
        sum += qv[q];
    }
    long long tot;
    long long A = tile_prefix[blockIdx.x] + block_excl_scan_ll(sum, tot) +
                  static_cast<long long>(U);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        const long long i = base + q;
        if (i >= N) break;
        const long long f = qv[q] >> 32;
        const unsigned long long p32 = static_cast<unsigned long long>(qv[q]) & 0xFFFFFFFFull;
        const unsigned long long a32 = static_cast<unsigned long long>(A) & 0xFFFFFFFFull;
        const bool extra = a32 + p32 >= (1ull << 32);
        const int n = static_cast<int>(f) + (extra ? 1 : 0);
        const int off = static_cast<int>(A >> 32);
        double wd = 1.0;
        if (extra && !hard) {
            const double u = __dmul_rn(static_cast<double>(a32), 0x1p-32);
            const double p = __dmul_rn(static_cast<double>(p32), 0x1p-32);
            const double r0 = __dmul_rn(__ddiv_rn(lam, p), __dsub_rn(__dadd_rn(u, p), 1.0));
            wd = __dmul_rn(h, r0 < 0.0 ? 0.0 : (r0 > 1.0 ? 1.0 : r0));
        }
        offsets[i] = off;
        if (counts) counts[i] = n;
        s_out[i] = valid ? __double2float_rn(__dadd_rn(a, __dmul_rn(c, static_cast<double>(d[i]))))
                         : 1.0f;
        w_out[i] = __double2float_rn(wd);
        for (int r = 0; r < n; ++r) {
            const long long t = static_cast<long long>(off) + r;
            if (t < capacity) sample_pixel[t] = static_cast<int32_t>(i);
        }
        A += qv[q];
        if (i == N - 1) {
            const long long T = A >> 32;
            offsets[N] = static_cast<int32_t>(T);
            *total = T;
            if (T > capacity) set_status(status, SPP_ERR_CAPACITY);
        }
    }
}

}  // namespace

size_t alloc_tiles(long long N) { return static_cast<size_t>((N + kTile - 1) / kTile); }

}  // namespace spp

extern "C" {

size_t spp_alloc_workspace_bytes(int W, int H) {
    if (W < 0 || H < 0) return 0;
    const long long N = static_cast<long long>(W) * H;
    return spp::kHeaderBytes + spp::alloc_tiles(N) * sizeof(unsigned long long);
}

}  // extern "C"

namespace spp {
namespace {
int alloc_impl(const float *d, int W, int H, const spp_params *p, const Dither &dither,
               int32_t *counts, int32_t *offsets, int32_t *sample_pixel, int64_t capacity,
               float *s_out, float *holdout_w, int64_t *total, int32_t *status, void *ws,
               size_t ws_bytes, cudaStream_t stream, bool systematic = false) {
    if (!p || W < 0 || H < 0 || capacity < 0) return SPP_ERR_ARG;
    if (static_cast<long long>(W) * H == 0) {  // empty frame: T = 0, offsets[0] = 0
        if (!offsets || !total) return SPP_ERR_ARG;
        if (!aligned16(offsets) || !aligned16(total)) return SPP_ERR_ALIGN;
        if (cudaMemsetAsync(offsets, 0, sizeof(int32_t), stream) != cudaSuccess) return SPP_ERR_CUDA;
        if (cudaMemsetAsync(total, 0, sizeof(int64_t), stream) != cudaSuccess) return SPP_ERR_CUDA;
        return SPP_OK;
    }
    if (!d || !offsets || !s_out || !holdout_w || !total || !status || !ws) return SPP_ERR_ARG;
    if (capacity > 0 && !sample_pixel) return SPP_ERR_ARG;
    if (!(p->budget > 0.0) || !(p->budget < 1e30)) return SPP_ERR_ARG;
    if (!(p->uniform_fraction >= 0.0) || !(p->uniform_fraction <= 1.0)) return SPP_ERR_ARG;
    if (p->holdout_mode != SPP_HOLDOUT_RAMP && p->holdout_mode != SPP_HOLDOUT_HARD &&
        p->holdout_mode != SPP_HOLDOUT_GUMBEL && p->holdout_mode != SPP_HOLDOUT_DASR)
        return SPP_ERR_ARG;
    if (p->holdout_mode == SPP_HOLDOUT_DASR && systematic) return SPP_ERR_ARG;
    if (p->holdout_mode == SPP_HOLDOUT_RAMP && !(p->lambda >= 1.0 && p->lambda < 1e30))
        return SPP_ERR_ARG;
    if (p->holdout_mode == SPP_HOLDOUT_GUMBEL &&
        (!(p->lambda > 0.0 && p->lambda < 1e30) || systematic))
        return SPP_ERR_ARG;
    if (p->reserved != 0 || (p->flags & ~(SPP_FLAG_EXACT_FP64 | SPP_FLAG_TEST_STALL_TILE1)) != 0)
        return SPP_ERR_ARG;
    const long long N = static_cast<long long>(W) * H;
    if (N >= (1ll << 31) - 1) return SPP_ERR_ARG;
    if (p->budget * static_cast<double>(N) + static_cast<double>(N) >= 2147483647.0)
        return SPP_ERR_ARG;
    if (!aligned16(d) || !aligned16(offsets) || !aligned16(s_out) || !aligned16(holdout_w) ||
        (counts && !aligned16(counts)) || !aligned16(ws) || !aligned16(total))
        return SPP_ERR_ALIGN;
    const size_t need = spp_alloc_workspace_bytes(W, H);
    if (ws_bytes < need) return SPP_ERR_WORKSPACE;

    if (cudaMemsetAsync(ws, 0, need, stream) != cudaSuccess) return SPP_ERR_CUDA;
    auto *hdr = static_cast<AllocHeader *>(ws);
    auto *tiles = reinterpret_cast<unsigned long long *>(static_cast<char *>(ws) + kHeaderBytes);

    BudgetArgs args;
    args.budget = p->budget;
    args.phi = p->uniform_fraction;
    const bool no_ramp = p->holdout_mode == SPP_HOLDOUT_HARD || p->holdout_mode == SPP_HOLDOUT_DASR;
    args.lambda = no_ramp ? 1.0 : p->lambda;
    args.hard = p->holdout_mode == SPP_HOLDOUT_HARD     ? 1
                : p->holdout_mode == SPP_HOLDOUT_GUMBEL ? kModeGumbel
                : p->holdout_mode == SPP_HOLDOUT_DASR   ? kModeDasr
                                                        : 0;
    // the Gumbel forward and the deterministic rounding decide every pixel in
    // FP64 (no float-float filter)
    args.force_exact =
        ((p->flags & SPP_FLAG_EXACT_FP64) || args.hard == kModeGumbel || args.hard == kModeDasr)
            ? 1
            : 0;

    // 8 values per thread and pass: enough blocks to fill every SM several
    // times over (the per-element carry chain is latency-bound)
    constexpr int kSumU = 2;
    const long long per_block = static_cast<long long>(kSumThreads) * 4 * kSumU;
    long long grid = (N + per_block - 1) / per_block;
    // up to eight blocks per SM.  Two per SM made the sample map alone faster
    // (38.5 against 40.6 us at 1080p, L2 flushed before each call) but the
    // 1080p frame slower (0.2093 against 0.2013 ms, three alternating runs on
    // one GPU): inside the frame the longer blocks start behind the previous
    // kernel's tail under programmatic dependent launch
    const long long max_grid = static_cast<long long>(sm_count()) * 8;
    if (grid > max_grid) grid = max_grid;
    if (grid < 1) grid = 1;
    launch_dependent(budget_sum_kernel<kSumU>, dim3(static_cast<unsigned>(grid)),
                     dim3(kSumThreads), 0, stream, d, N, hdr, args, status);
    const int num_tiles = static_cast<int>(alloc_tiles(N));
    if (systematic) {
        // the frame offset U: the top 32 bits of element 2^62 of the stream
        const unsigned long long U =
            stream_bits(stream_key(p->seed, p->frame), 1ull << 62) >> 32;
        auto *tile_sums = reinterpret_cast<long long *>(tiles);
        sys_tile_sum_kernel<<<num_tiles, kScanThreads, 0, stream>>>(d, N, hdr, tile_sums);
        sys_scan_tiles_kernel<<<1, kScanThreads, 0, stream>>>(tile_sums, num_tiles);
        sys_assign_kernel<<<num_tiles, kScanThreads, 0, stream>>>(
            d, N, hdr, tile_sums, U, args.hard, counts, offsets, sample_pixel, capacity, s_out,
            holdout_w, reinterpret_cast<long long *>(total), status);
        count_launch(4);
        return launch_status();
    }
    Dither dt = dither;
    dt.W = W;
    const bool stall = (p->flags & SPP_FLAG_TEST_STALL_TILE1) != 0;
    if (num_tiles > kSinglePassMaxTiles && counts && !stall) {
        auto *tile_sums = reinterpret_cast<int *>(tiles);
        launch_dependent(assign_tile_kernel, dim3(num_tiles), dim3(kScanThreads), 0, stream, d,
                         N, hdr, stream_key(p->seed, p->frame), dt, args.hard, counts, s_out,
                         holdout_w, tile_sums);
        launch_dependent(offsets_kernel, dim3(num_tiles), dim3(kScanThreads), 0, stream, counts,
                         N, tile_sums, num_tiles, offsets, sample_pixel, capacity,
                         reinterpret_cast<long long *>(total), status);
        count_launch(3);
        return launch_status();
    }
    launch_dependent(assign_scan_kernel, dim3(num_tiles), dim3(kScanThreads), 0, stream, d, N,
                     hdr, hdr, tiles, stream_key(p->seed, p->frame), dt, args.hard,
                     (p->flags & SPP_FLAG_TEST_STALL_TILE1) ? 1 : 0, counts, offsets,
                     sample_pixel, capacity, s_out, holdout_w,
                     reinterpret_cast<long long *>(total), status, num_tiles);
    count_launch(2);
    return launch_status();
}
}  // namespace
}  // namespace spp

extern "C" {

int spp_alloc_sample_map(const float *d, int W, int H, const spp_params *p, int32_t *counts,
                         int32_t *offsets, int32_t *sample_pixel, int64_t capacity, float *s_out,
                         float *holdout_w, int64_t *total, int32_t *status, void *ws,
                         size_t ws_bytes, cudaStream_t stream) {
    return spp::alloc_impl(d, W, H, p, spp::Dither{}, counts, offsets, sample_pixel, capacity,
                           s_out, holdout_w, total, status, ws, ws_bytes, stream);
}

int spp_alloc_sample_map_systematic(const float *d, int W, int H, const spp_params *p,
                                    int32_t *counts, int32_t *offsets, int32_t *sample_pixel,
                                    int64_t capacity, float *s_out, float *holdout_w,
                                    int64_t *total, int32_t *status, void *ws, size_t ws_bytes,
                                    cudaStream_t stream) {
    if (p && (p->flags & SPP_FLAG_TEST_STALL_TILE1)) return SPP_ERR_ARG;
    return spp::alloc_impl(d, W, H, p, spp::Dither{}, counts, offsets, sample_pixel, capacity,
                           s_out, holdout_w, total, status, ws, ws_bytes, stream, true);
}

int spp_alloc_sample_map_dithered(const float *d, int W, int H, const spp_params *p,
                                  const uint16_t *mask, int T, int32_t *counts, int32_t *offsets,
                                  int32_t *sample_pixel, int64_t capacity, float *s_out,
                                  float *holdout_w, int64_t *total, int32_t *status, void *ws,
                                  size_t ws_bytes, cudaStream_t stream) {
    using namespace spp;
    if (!mask || !p) return SPP_ERR_ARG;
    if (T < 4 || T > 256 || (T & (T - 1))) return SPP_ERR_ARG;
    if (!aligned16(mask)) return SPP_ERR_ALIGN;
    Dither dt;
    dt.mask = mask;
    dt.log2T = 0;
    while ((1 << dt.log2T) < T) ++dt.log2T;
    dt.off48 = (static_cast<uint64_t>(p->frame) * (kGamma >> 16) + (mix64(p->seed) >> 16)) &
               0xFFFFFFFFFFFFull;
    return alloc_impl(d, W, H, p, dt, counts, offsets, sample_pixel, capacity, s_out, holdout_w,
                      total, status, ws, ws_bytes, stream);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of spp_alloc_sample_map.
//
// Some callers cannot allocate device memory while they run: an engine or
// plug-in host that owns the GPU's memory budget and forbids allocation inside
// its frame loop (cudaMalloc can synchronise the device and its latency is
// unbounded).  This entry point therefore keeps its scratch (the budget-sum
// header and the scan's tile states) in a library-owned array in device memory
// instead of a caller workspace.  The array has a fixed size, so frames are
// limited to kStaticMaxPixels pixels; every GPU that loads the library keeps
// it resident until the process exits.
// ---------------------------------------------------------------------------
namespace spp {
namespace {
constexpr long long kStaticMaxPixels = 1ll << 25;  // 33,554,432 pixels (8K UHD fits)
constexpr size_t kStaticScratchBytes =
    kHeaderBytes + static_cast<size_t>((kStaticMaxPixels + kTile - 1) / kTile) *
                       sizeof(unsigned long long);  // 131,328 bytes
}  // namespace
}  // namespace spp

static __device__ __align__(256) unsigned char spp_static_scratch[spp::kStaticScratchBytes];

namespace spp {
namespace {
// The host-side name spp_static_scratch is only a stand-in for the array; its
// device address is looked up once per device, with that device current.
void *static_scratch_address(int *rc) {
    static std::mutex mu;
    constexpr int kMaxDevices = 64;
    static void *addr[kMaxDevices] = {nullptr};
    // a failed runtime call's error is taken off the thread's error state
    // here, so that this call reports it and the next, unrelated call does not
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        *rc = SPP_ERR_CUDA;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, spp_static_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            *rc = SPP_ERR_CUDA;
            return nullptr;
        }
        addr[dev] = p;
    }
    return addr[dev];
}
}  // namespace
}  // namespace spp

extern "C" int spp_alloc_sample_map_static(const float *d, int W, int H, const spp_params *p,
                                           int32_t *counts, int32_t *offsets,
                                           int32_t *sample_pixel, int64_t capacity, float *s_out,
                                           float *holdout_w, int64_t *total, int32_t *status,
                                           cudaStream_t stream) {
    using namespace spp;
    if (W < 0 || H < 0) return SPP_ERR_ARG;
    if (static_cast<long long>(W) * H > kStaticMaxPixels) return SPP_ERR_WORKSPACE;
    int rc = SPP_OK;
    void *ws = static_scratch_address(&rc);
    if (!ws) return rc;
    // the regular entry point clears the header and tile states it uses before
    // its kernels run, so leftovers of the previous call do not matter
    return spp_alloc_sample_map(d, W, H, p, counts, offsets, sample_pixel, capacity, s_out,
                                holdout_w, total, status, ws, kStaticScratchBytes, stream);
}
