"""Oracles of the pipeline variants of Sec. 7 (ablations): the
low-resolution density map and the systematic (exact-integer-total)
rounding of the sample map.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests,
``__graft_entry__.smoke()`` and the CPU baseline leg of ``bench.py`` call it;
the product never imports it.

Low-resolution density (Sec. 7, the density predicted at full resolution is
brought to a quarter of the pixels before the stochastic sampling).  Reading:
P = nearest upsampling of the f x f block means (f = 2: a quarter of the
pixels), applied to the density before the budget normalisation.  P is a
symmetric projection (block-constant images are fixed, <P a, b> = <a, P b>),
so the same map takes the gradient with respect to P d back to d.  The block
mean is summed in FP32 as a pairwise tree (each row of the block: adjacent
pairs, then pairs of pairs; then the row sums the same way, top to bottom)
and scaled by 1/f^2 (exact), so the GPU reproduces it bit for bit and a
block-constant image is an exact fixed point.

Systematic rounding (the exact-integer-total reading of the budget of Sec. 3:
the realised sample count is fixed to within one sample instead of varying
by about sqrt(B N)).  Every pixel's interval of length s_i is laid end to end
on one line, shifted by one frame offset U; pixel i receives the integers
its interval covers.  In 32.32 fixed point, exactly and independently of
the summation order:
  q_i = round-to-nearest-even(s_i 2^32)       (s_i of Sec. 3, FP64)
  P_i = q_0 + ... + q_i (P_-1 = 0),  A_i = P_{i-1} + U,  U in [0, 2^32)
  offsets_i = floor(A_i / 2^32),  n_i = offsets_{i+1} - offsets_i,
  T = floor((P_{N-1} + U) / 2^32)
so n_i = f_i + extra_i with f_i = floor(q_i / 2^32) and extra_i iff
a_i + p_i >= 1, a_i = (A_i mod 2^32) 2^-32, p_i = (q_i mod 2^32) 2^-32: the
stochastic test of Sec. 4.2 with u_i replaced by the position a_i of the
pixel's interval on the integer grid (over a uniform U, E[n_i] = q_i 2^-32).
The holdout weight of an extra sample is the relaxed ramp of Sec. 4.3 at
u = a_i (h, lambda as for the stochastic map; hard mode: 1).
U = the top 32 bits of element 2^62 of the SplitMix64 stream of
(seed, frame) (key = mix(seed + (frame + 1) gamma), element i = mix(key +
(i + 1) gamma)).

Gradient estimators of the discretisation (the ablation of Sec. 7 that
compares the relaxed ramp of Sec. 4.3 with the straight-through estimator,
Bengio et al. 2013, and the Gumbel-softmax / binary concrete relaxation,
Jang et al. 2017, Maddison et al. 2017), with L^0 = (sum_{k<f} S_k +
e w S_f) / s per pixel (Eq. stoch_rnoisy), f = floor(s), p = s - f:
  straight-through  forward: the hard rule e = [u > 1 - p], w = 1; backward:
                    de/dp := 1, so dL^0/ds = (S_f - L^0) / s, where S_f is the
                    sample of slot f, rendered for the gradient when the
                    forward did not trace it (the paper trains on
                    pre-rendered samples, so every slot exists)
  Gumbel-softmax    forward (training): the extra sample is always traced
                    (p > 0) with weight w = sigma(lambda (ln(p / (1 - p)) +
                    ln(u / (1 - u)))), lambda the inverse temperature;
                    backward: dw/dp = lambda w (1 - w) / (p (1 - p)); at test
                    time the hard rule, w > 1/2 iff u > 1 - p
  DASR              the deterministic rounding of Sec. 4.1 (Eq. kuz_fw,
                    after Kuznetsov et al. 2018): n = round(s) samples,
                    L^0 = (sum_{j<n} S_j) / n for s >= 1/2, else 0; its
                    surrogate gradient (Eq. kuz_grad) dL^0/ds = (L^ref - L^0)
                    / round(s) for s >= 1/2, else L^ref, with L^ref the
                    reference radiance of the pixel.  round() takes halves
                    up (n = floor(s) + [s - floor(s) >= 1/2]): the equation's
                    branch s >= 1/2 divides by round(s), which must then be at
                    least one.  The same rule serves training and test time.

Pins (tests/test_oracle_variants_pins.py): block-constant images are fixed
points, the sum is preserved (FP64), symmetry, agreement with a library
reshape-mean, and the density gradient through P against finite
differences; for the systematic map the total within one sample of B N,
unbiasedness over all offsets U on a grid, evenly spaced samples for a
constant density, and agreement with the C oracle's independent stochastic
assignment at u = a_i; for the estimators: the Gumbel relaxation's gradient
against finite differences of its forward, its hard limit (lambda -> inf) is
the stochastic map, and the straight-through gradient against its closed
form on one pixel; for DASR hand-computed counts at and around the
half-integers, |n - s| <= 1/2 with exact rational arithmetic, the forward's
sample mean and its zero below the threshold, the budget's total within N/2,
and hand-computed surrogate gradients on both sides of the threshold.
"""
from __future__ import annotations

import numpy as np


def density_lowres(d, W: int, H: int, factor: int) -> np.ndarray:
    """P d for d [H*W] (or [H][W]) FP32; returns FP32 [H*W]."""
    f = int(factor)
    d = np.asarray(d, np.float32).reshape(H, W)
    if f not in (1, 2, 4, 8) or H % f or W % f:
        raise ValueError("factor 1, 2, 4 or 8 dividing W and H")
    def tree(parts):
        while len(parts) > 1:
            parts = [(parts[k] + parts[k + 1]).astype(np.float32) for k in range(0, len(parts), 2)]
        return parts[0]

    rows = [tree([d[r::f, c::f] for c in range(f)]) for r in range(f)]
    mean = (tree(rows) * np.float32(1.0 / (f * f))).astype(np.float32)
    return np.repeat(np.repeat(mean, f, axis=0), f, axis=1).reshape(-1)


# ------------------------------------------------------ systematic rounding
M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def _mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def systematic_offset(seed: int, frame: int) -> int:
    key = _mix((seed + (frame + 1) * GAMMA) & M64)
    return _mix((key + ((1 << 62) + 1) * GAMMA) & M64) >> 32


class SystematicAlloc:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def alloc_systematic(d, B: float, phi: float = 0.125, lam: float = 10.0, hard: bool = False,
                     seed: int = 0x5EED, frame: int = 0, U: int | None = None):
    """Systematic sample map of the FP32 density d [N] (Sec. 3 budget)."""
    import oracle
    rc, S, a, c = oracle.budget_coeffs(d, B, phi)
    if rc != 0:
        raise ValueError(f"budget rc={rc}")
    d64 = np.asarray(d, np.float32).astype(np.float64).ravel()
    s = a + c * d64                                   # FP64, product then sum
    q = np.rint(np.ldexp(s, 32)).astype(np.int64)    # ties to even
    if U is None:
        U = systematic_offset(seed, frame)
    P = np.concatenate([[0], np.cumsum(q)]).astype(np.int64)
    A = P[:-1] + np.int64(U)
    offsets = np.concatenate([A >> 32, [(P[-1] + np.int64(U)) >> 32]]).astype(np.int64)
    f = q >> 32
    p32 = q & 0xFFFFFFFF
    a32 = A & 0xFFFFFFFF
    extra = (a32 + p32) >= (1 << 32)
    n = f + extra
    assert np.array_equal(np.diff(offsets), n)
    w = np.ones(d64.size)
    if not hard:
        h = (2.0 * lam) / (2.0 * lam - 1.0)
        idx = np.flatnonzero(extra)
        u = a32[idx].astype(np.float64) * 2.0 ** -32
        pp = p32[idx].astype(np.float64) * 2.0 ** -32
        r = (lam / pp) * ((u + pp) - 1.0)
        w[idx] = h * np.clip(r, 0.0, 1.0)
    return SystematicAlloc(counts=n, offsets=offsets, s=s, q=q, U=U, a32=a32, extra=extra,
                           w=w.astype(np.float32), T=int(offsets[-1]))


# ------------------------------------------------ gradient estimators
def gumbel_weight(p, u, lam):
    """sigma(lam (ln(p / (1 - p)) + ln(u / (1 - u)))), FP64."""
    p = np.asarray(p, np.float64)
    u = np.asarray(u, np.float64)
    with np.errstate(divide="ignore", over="ignore"):
        x = lam * (np.log(p / (1.0 - p)) + np.log(u / (1.0 - u)))
        return 1.0 / (1.0 + np.exp(-x))


def alloc_gumbel(d, B: float, phi: float = 0.125, lam: float = 10.0, seed: int = 0x5EED,
                 frame: int = 0):
    """Training-time sample map of the Gumbel-softmax estimator: every pixel
    with p > 0 gets its extra sample, weighted by the relaxed indicator."""
    import oracle
    rc, S, a, c = oracle.budget_coeffs(d, B, phi)
    if rc != 0:
        raise ValueError(f"budget rc={rc}")
    d64 = np.asarray(d, np.float32).astype(np.float64).ravel()
    s = a + c * d64
    f = np.floor(s)
    p = s - f
    u = np.array([oracle.pixel_uniform(seed, frame, i) for i in range(s.size)])
    extra = p > 0.0
    n = f.astype(np.int64) + extra
    w = np.where(extra, gumbel_weight(np.where(extra, p, 0.5), u, lam), 1.0)
    offsets = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    return SystematicAlloc(counts=n, offsets=offsets, s=s, w=w.astype(np.float32), extra=extra,
                           u=u, p=p, T=int(offsets[-1]))


def splat_backward_estimator(a, rgb, L0, grad_L0, estimator: str, lam: float = 10.0,
                             clean=None, render_seed: int = 0, frame: int = 0) -> np.ndarray:
    """dLoss/ds of the splat under the straight-through or Gumbel-softmax
    estimator; a: the allocation (counts, offsets, s, extra; for Gumbel its
    weights w and p), rgb [T][3] the traced samples."""
    import oracle
    rgb = np.asarray(rgb, np.float64).reshape(-1, 3)
    L0 = np.asarray(L0, np.float64).reshape(3, -1)
    g = np.asarray(grad_L0, np.float64).reshape(3, -1)
    s = np.asarray(a.s, np.float64)
    N = s.size
    out = -(g * L0).sum(axis=0) / s
    if estimator == "gumbel":
        for i in np.flatnonzero(a.extra):
            w = float(a.w[i])
            p = float(a.p[i])
            dw = lam * w * (1.0 - w) / (p * (1.0 - p))
            S = rgb[a.offsets[i + 1] - 1]
            out[i] += float(g[:, i] @ S) * dw / s[i]
    elif estimator == "straight_through":
        clean = np.asarray(clean, np.float64).reshape(3, -1)
        for i in range(N):
            f = int(np.floor(s[i]))
            if s[i] - f <= 0.0:
                continue
            if a.counts[i] > f:
                S = rgb[a.offsets[i + 1] - 1]
            else:  # the untraced sample of slot f
                S = clean[:, i] * oracle.sample_noise(render_seed, frame, i, f)
            out[i] += float(g[:, i] @ S) / s[i]
    else:
        raise ValueError(estimator)
    return out


# ------------------------------------- DASR: deterministic rounding (Sec. 4.1)
def dasr_counts(s) -> np.ndarray:
    """n_i = round(s_i) of Eq. kuz_fw, halves up: floor(s) + [s - floor(s) >= 1/2]
    (s - floor(s) is exact in FP64, so the comparison is exact)."""
    s = np.asarray(s, np.float64)
    f = np.floor(s)
    return (f + ((s - f) >= 0.5)).astype(np.int64)


def alloc_dasr(d, B: float, phi: float = 0.125):
    """Deterministic sample map of the FP32 density d [N]: the s_i of the
    budget normalisation (Sec. 3), n_i = round(s_i), offsets, and the
    normaliser of Eq. kuz_fw, max(n_i, 1) (a pixel without samples has
    L^0 = 0 whatever it is divided by)."""
    import oracle
    rc, S, a, c = oracle.budget_coeffs(d, B, phi)
    if rc != 0:
        raise ValueError(f"budget rc={rc}")
    d64 = np.asarray(d, np.float32).astype(np.float64).ravel()
    s = a + c * d64                                   # FP64, product then sum
    n = dasr_counts(s)
    offsets = np.concatenate([[0], np.cumsum(n)]).astype(np.int64)
    return SystematicAlloc(counts=n, offsets=offsets, s=s, norm=np.maximum(n, 1),
                           T=int(offsets[-1]))


def splat_dasr(counts, rgb, W: int, H: int, L: int) -> list[np.ndarray]:
    """Eq. kuz_fw per pixel, L^0_i = (sum_{j<n_i} S_ij) / n_i (0 when n_i = 0),
    with the samples of pixel i consecutive in rgb [T][3] (pixel order), then
    the 2^l x 2^l block means of Eq. app-pyramid."""
    n = np.asarray(counts, np.int64).ravel()
    rgb = np.asarray(rgb, np.float64).reshape(-1, 3)
    offsets = np.concatenate([[0], np.cumsum(n)])
    L0 = np.zeros((W * H, 3))
    for i in np.flatnonzero(n):
        L0[i] = rgb[offsets[i]:offsets[i + 1]].sum(axis=0) / n[i]
    L0 = L0.T.reshape(3, H, W)
    layers = [L0]
    for l in range(1, L):
        f = 1 << l
        layers.append(L0.reshape(3, H // f, f, W // f, f).mean(axis=(2, 4)))
    return layers


def splat_backward_dasr(counts, L0, grad_L0, ref) -> np.ndarray:
    """dLoss/ds_i through Eq. kuz_grad: sum_c g_ic (L^ref_ic - L^0_ic) / n_i
    where n_i = round(s_i) >= 1 (s_i >= 1/2), else sum_c g_ic L^ref_ic."""
    n = np.asarray(counts, np.int64).ravel()
    L0 = np.asarray(L0, np.float64).reshape(3, -1)
    g = np.asarray(grad_L0, np.float64).reshape(3, -1)
    ref = np.asarray(ref, np.float64).reshape(3, -1)
    sampled = (g * (ref - L0)).sum(axis=0) / np.maximum(n, 1)
    return np.where(n >= 1, sampled, (g * ref).sum(axis=0))
