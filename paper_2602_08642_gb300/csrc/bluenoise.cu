// Blue-noise dither mask for the discretisation of the sampling density
// (Sec. 6.3 dithers with blue noise, after Ulichney's void-and-cluster
// method, 1993).  Host code: the mask is generated once and uploaded; the
// allocation kernel tiles it over the frame.
//
// The method on a T x T torus (T a power of two), Gaussian filter sigma 1.5:
//  - filter weights are integers, round(2^20 exp(-r^2 / (2 sigma^2))) with the
//    toroidal distance r, so every energy is an exact integer sum and the
//    result does not depend on the order of any accumulation;
//  - the energy of a pixel is the weighted count of set pixels around it; the
//    tightest cluster is the set pixel of largest energy, the largest void
//    the unset pixel of smallest energy (ties: the smallest index y T + x);
//  - start pattern: floor(T^2 / 10) pixels at the first distinct positions
//    SplitMix64(seed) mod T^2;
//  - prototype: move the tightest cluster into the largest void until the
//    two coincide;
//  - ranks: removing clusters from the prototype one by one gives ranks
//    ones-1 .. 0; filling voids from the prototype gives ones .. T^2-1 (for
//    a linear energy the method's phase of "clusters of zeros" is the same
//    void filling).
#include <cmath>
#include <cstdint>
#include <vector>

#include "spp_internal.cuh"

namespace spp {
namespace {

struct Torus {
    int T;
    std::vector<int64_t> w;  // w[dy * T + dx]
    explicit Torus(int t) : T(t), w(static_cast<size_t>(t) * t) {
        for (int dy = 0; dy < T; ++dy)
            for (int dx = 0; dx < T; ++dx) {
                const int ey = dy < T - dy ? dy : T - dy, ex = dx < T - dx ? dx : T - dx;
                const double g = std::exp(-static_cast<double>(ex * ex + ey * ey) / (2.0 * 1.5 * 1.5));
                w[static_cast<size_t>(dy) * T + dx] = static_cast<int64_t>(std::floor(1048576.0 * g + 0.5));
            }
    }
    // E += sign * (weights of every pixel relative to pixel q)
    void add(std::vector<int64_t> &E, int q, int64_t sign) const {
        const int qy = q / T, qx = q % T;
        for (int y = 0; y < T; ++y) {
            const int64_t *row = &w[static_cast<size_t>((y - qy) & (T - 1)) * T];
            int64_t *e = &E[static_cast<size_t>(y) * T];
            for (int x = 0; x < T; ++x) e[x] += sign * row[(x - qx) & (T - 1)];
        }
    }
};

int tightest_cluster(const std::vector<uint8_t> &P, const std::vector<int64_t> &E) {
    int best = -1;
    for (size_t i = 0; i < P.size(); ++i)
        if (P[i] && (best < 0 || E[i] > E[best])) best = static_cast<int>(i);
    return best;
}

int largest_void(const std::vector<uint8_t> &P, const std::vector<int64_t> &E) {
    int best = -1;
    for (size_t i = 0; i < P.size(); ++i)
        if (!P[i] && (best < 0 || E[i] < E[best])) best = static_cast<int>(i);
    return best;
}

}  // namespace
}  // namespace spp

extern "C" int spp_blue_noise_mask(int T, uint64_t seed, uint16_t *rank) {
    using namespace spp;
    if (!rank || T < 4 || T > 256 || (T & (T - 1))) return SPP_ERR_ARG;
    const int n = T * T;
    const Torus tor(T);
    std::vector<uint8_t> P(n, 0);
    std::vector<int64_t> E(n, 0);
    const int ones = n / 10;
    uint64_t state = seed;
    for (int placed = 0; placed < ones;) {
        state += kGamma;
        const int i = static_cast<int>(mix64(state) % static_cast<uint64_t>(n));
        if (!P[i]) {
            P[i] = 1;
            tor.add(E, i, 1);
            ++placed;
        }
    }
    for (int it = 0; it < n; ++it) {  // prototype
        const int c = tightest_cluster(P, E);
        P[c] = 0;
        tor.add(E, c, -1);
        const int v = largest_void(P, E);
        if (v == c) {
            P[c] = 1;
            tor.add(E, c, 1);
            break;
        }
        P[v] = 1;
        tor.add(E, v, 1);
    }
    std::vector<uint8_t> Q = P;
    std::vector<int64_t> EQ = E;
    for (int r = ones - 1; r >= 0; --r) {
        const int c = tightest_cluster(Q, EQ);
        rank[c] = static_cast<uint16_t>(r);
        Q[c] = 0;
        tor.add(EQ, c, -1);
    }
    Q = P;
    EQ = E;
    for (int r = ones; r < n; ++r) {
        const int v = largest_void(Q, EQ);
        rank[v] = static_cast<uint16_t>(r);
        Q[v] = 1;
        tor.add(EQ, v, 1);
    }
    return SPP_OK;
}
