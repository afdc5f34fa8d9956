"""Oracle of the blue-noise dithering of the discretisation (Sec. 6.3: the
stochastic rounding of Sec. 4.2 takes its uniforms from a blue-noise mask,
after Ulichney's void-and-cluster method, 1993).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

The mask is a T x T rank matrix (a permutation of 0 .. T^2 - 1, T a power of
two), tiled over the frame.  Generation, written from the published method
(void-and-cluster, toroidal Gaussian energy with sigma = 1.5):

  weights   w(dx, dy) = round(2^20 exp(-(dx'^2 + dy'^2) / (2 sigma^2))) with
            dx' = min(dx mod T, T - dx mod T), likewise dy' (integers, so
            every energy below is an exact integer sum, independent of order)
  energy    E(p) = sum over set pixels q of w(p - q)
  cluster   the set pixel of largest E; void: the unset pixel of smallest E;
            ties go to the smallest index y T + x
  start     floor(T^2 / 10) pixels set at the first distinct positions
            (SplitMix64 output of the seed) mod T^2
  prototype repeat at most T^2 times: remove the tightest cluster c; find the
            largest void v; if v == c put it back and stop, else set v
  phase 1   from the prototype, remove tightest clusters one by one; the
            k-th removed gets rank (ones - k)
  phase 2   from the prototype, fill largest voids one by one; they get ranks
            ones, ones + 1, ... up to T^2 - 1 (for a linear energy the
            "tightest cluster of zeros" of the method's third phase is the
            largest void, so phases 2 and 3 are one loop)

Uniform of pixel (x, y) in frame t (48-bit fixed point, exact):
  u48 = (rank[y mod T][x mod T] 2^(48 - 2k) + 2^(47 - 2k)
         + t G48 + (mix(seed) >> 16)) mod 2^48,   T = 2^k,
  G48 = the top 48 bits of the golden-ratio gamma 0x9E3779B97F4A7C15, mix =
  the SplitMix64 finaliser; u = u48 2^-48.  Within a tile the uniforms of a
  frame are the stratified values (r + 1/2) / T^2 in blue-noise order; the
  golden-ratio step moves every pixel's threshold between frames.
"""
from __future__ import annotations

import math

import numpy as np

SIGMA = 1.5
GAMMA = 0x9E3779B97F4A7C15
G48 = GAMMA >> 16
M64 = (1 << 64) - 1


def _mix(z: int) -> int:
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 & M64
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB & M64
    return z ^ (z >> 31)


def weights(T: int) -> np.ndarray:
    """Integer toroidal Gaussian kernel w[dy][dx]."""
    w = np.empty((T, T), np.int64)
    for dy in range(T):
        ey = min(dy, T - dy)
        for dx in range(T):
            ex = min(dx, T - dx)
            w[dy, dx] = int(math.floor(2.0 ** 20 * math.exp(-(ex * ex + ey * ey) / (2.0 * SIGMA * SIGMA)) + 0.5))
    return w


def mask(T: int, seed: int) -> np.ndarray:
    """The T x T rank matrix (uint16)."""
    if T < 4 or T & (T - 1) or T > 256:
        raise ValueError("T must be a power of two in [4, 256]")
    n = T * T
    wt = weights(T)

    def kern(p):  # weights of every pixel relative to pixel p, flattened
        py, px = divmod(p, T)
        return np.roll(np.roll(wt, py, axis=0), px, axis=1).ravel()

    P = np.zeros(n, bool)
    ones = n // 10
    state = seed & M64
    placed = 0
    while placed < ones:
        state = (state + GAMMA) & M64
        i = _mix(state) % n
        if not P[i]:
            P[i] = True
            placed += 1
    E = np.zeros(n, np.int64)
    for p in np.flatnonzero(P):
        E += kern(int(p))

    big = np.int64(1) << 62

    def cluster(P, E):
        return int(np.argmax(np.where(P, E, -big)))

    def void(P, E):
        return int(np.argmin(np.where(P, big, E)))

    for _ in range(n):
        c = cluster(P, E)
        P[c] = False
        E -= kern(c)
        v = void(P, E)
        if v == c:
            P[c] = True
            E += kern(c)
            break
        P[v] = True
        E += kern(v)

    rank = np.empty(n, np.int64)
    Q, EQ = P.copy(), E.copy()
    for r in range(ones - 1, -1, -1):
        c = cluster(Q, EQ)
        rank[c] = r
        Q[c] = False
        EQ -= kern(c)
    Q, EQ = P.copy(), E.copy()
    for r in range(ones, n):
        v = void(Q, EQ)
        rank[v] = r
        Q[v] = True
        EQ += kern(v)
    return rank.reshape(T, T).astype(np.uint16)


def uniform48(rank: np.ndarray, W: int, H: int, seed: int, frame: int) -> np.ndarray:
    """u48 of every pixel of a W x H frame, flat in row-major order (uint64)."""
    T = rank.shape[0]
    k = T.bit_length() - 1
    off = (frame * G48 + (_mix(seed & M64) >> 16)) % (1 << 48)
    ys, xs = np.mgrid[0:H, 0:W]
    r = rank[ys % T, xs % T].astype(np.uint64).ravel()
    base = (r << np.uint64(48 - 2 * k)) + np.uint64(1 << (47 - 2 * k))
    return ((base + np.uint64(off)) & np.uint64((1 << 48) - 1)).astype(np.uint64)
