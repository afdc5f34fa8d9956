"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here reads the CUDA path.  Each test pins one oracle function to
something other than itself: a published test vector, a library routine
(math.fsum, fractions, scipy), a closed form the paper states, an invariant,
or brute force over a grid.  Every test names the passage it follows.
"""
import fractions
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# Counter-based generator (SplitMix64)
# ---------------------------------------------------------------------------
def test_splitmix64_reference_sequences(orc):
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    assert rows
    for row in rows:
        seed, outs = int(row[0]), [int(x) for x in row[1:]]
        assert orc.splitmix64_sequence(seed, len(outs)) == outs


def test_pixel_uniform_range_and_moments(orc):
    u = np.array([orc.pixel_uniform(0x5EED, 3, i) for i in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    # mean 1/2, variance 1/12 of U(0,1); 5 sigma bounds
    n = u.size
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * math.sqrt(1 / 180 / n)
    # values are multiples of 2^-48
    assert all(float(x * 2**48).is_integer() for x in u[:100])


# ---------------------------------------------------------------------------
# a1: exact budget sum (Sec. 3) -- correctly rounded, order independent
# ---------------------------------------------------------------------------
def _adversarial_f32(rng, n):
    e = rng.integers(-149, 127, size=n)
    m = rng.random(n)
    v = np.ldexp(1.0 + m, e).astype(np.float32)
    v[rng.random(n) < 0.05] = np.float32(1.4e-45)  # smallest subnormal
    v[rng.random(n) < 0.02] = np.float32(3.0e38)
    return v


def test_exact_sum_matches_fsum_and_fractions(orc):
    rng = np.random.default_rng(7)
    cases = [
        np.exp(rng.standard_normal(50000)).astype(np.float32),
        _adversarial_f32(rng, 4000),
        np.array([1.0, 2.0**-24, 2.0**-24], np.float32),       # half-way tie cases
        np.array([2.0**100, 1.0, 2.0**-100, 2.0**-149], np.float32),
        np.zeros(5, np.float32),
    ]
    for v in cases:
        ref = math.fsum(v.astype(np.float64).tolist())
        assert orc.exact_sum_f32(v) == ref
    for v in cases[1:]:
        exact = sum((fractions.Fraction(float(x)) for x in v), fractions.Fraction(0))
        assert orc.exact_sum_f32(v) == float(exact)


def test_exact_sum_permutation_invariant(orc):
    rng = np.random.default_rng(8)
    v = _adversarial_f32(rng, 3000)
    s0 = orc.exact_sum_f32(v)
    for _ in range(5):
        assert orc.exact_sum_f32(rng.permutation(v)) == s0


def test_budget_conserved_and_floor(orc):
    """Sec. 3: sum_i s_i = B N (1/8 uniform + 7/8 softmax), s_i >= B/8."""
    rng = np.random.default_rng(9)
    for B in (0.11, 0.25, 0.5, 4.0):
        d = np.exp(rng.standard_normal(4096)).astype(np.float32)
        a = orc.alloc(d, B)
        N = d.size
        total = orc.exact_sum_f64(a.s)
        assert abs(total - B * N) <= 4 * N * 2.0**-52 * B * N
        assert a.s.min() >= B / 8
        assert a.a == B / 8


def test_budget_scale_invariance_and_uniform(orc):
    """The softmax normalisation makes s invariant to scaling d by 2^k, and a
    constant d spreads the budget uniformly (s_i = B)."""
    rng = np.random.default_rng(10)
    d = np.exp(rng.standard_normal(1000)).astype(np.float32)
    a1 = orc.alloc(d, 0.25)
    a2 = orc.alloc(d * np.float32(8.0), 0.25)
    assert np.array_equal(a1.s, a2.s)
    c = orc.alloc(np.full(1000, 3.0, np.float32), 0.25)
    assert np.allclose(c.s, 0.25, rtol=4e-16, atol=0)


def test_budget_rejects_bad_density(orc):
    for bad in (np.array([1.0, -1.0], np.float32), np.array([1.0, np.nan], np.float32),
                np.array([1.0, np.inf], np.float32), np.zeros(4, np.float32)):
        assert orc.budget_coeffs(bad, 0.25)[0] == orc.ERR_INPUT


# ---------------------------------------------------------------------------
# a2: stochastic rounding and the relaxed ramp (Sec. 4.2-4.3)
# ---------------------------------------------------------------------------
M = 2**14
UGRID = (np.arange(M) + 0.5) / M


@pytest.mark.parametrize("s", [0.03125, 0.3, 0.5, 0.77, 1.3, 2.95, 7.5])
def test_extra_probability_and_unbiased_ramp(orc, s):
    """P(extra) = p (Sec. 4.2); E[H] over u equals p, so the ramp with the
    factor h = 2 lam/(2 lam - 1) keeps the holdout unbiased (Eq. h_factor);
    the linear region has probability p/lam (Sec. 4.3)."""
    lam = 10.0
    f = math.floor(s)
    p = s - f
    n_extra = 0
    w_sum = 0.0
    n_linear = 0
    for u in UGRID:
        n, w, e = orc.assign_one(s, float(u), lam)
        assert n in (f, f + 1) and n == f + e
        if e:
            n_extra += 1
            w_sum += w
            if w < 2 * lam / (2 * lam - 1):
                n_linear += 1
    assert abs(n_extra / M - p) <= 1.0 / M
    # midpoint rule on a piecewise-linear ramp: exact up to the two kink cells
    assert abs(w_sum / M - p) <= 2.0 * (2 * lam / (2 * lam - 1)) / M
    assert abs(n_linear / M - p / lam) <= 2.0 / M


def test_ramp_closed_form_points(orc):
    """Eq. relaxed_holdout at its characteristic points: 0 at u = 1-p, h/2 at
    the middle of the linear region, h above it."""
    lam, p = 10.0, 0.4
    h = 2 * lam / (2 * lam - 1)
    _, w, e = orc.assign_one(p, 1 - p + p / (2 * lam), lam)
    assert e == 1 and abs(w - h / 2) < 1e-12
    _, w, e = orc.assign_one(p, 0.999, lam)
    assert e == 1 and w == h
    _, w, e = orc.assign_one(p, 1 - p - 1e-9, lam)
    assert e == 0
    # the derivative on the linear region, dH/dp = h lam (1-u)/p^2
    u = 1 - p + p / (3 * lam)
    dp = 1e-7
    wp = orc.assign_one(p + dp, u, lam)[1]
    wm = orc.assign_one(p - dp, u, lam)[1]
    assert abs((wp - wm) / (2 * dp) - h * lam * (1 - u) / p**2) < 1e-5


def test_hard_limit(orc):
    """lam -> infinity recovers the hard step of Eq. holdout (Sec. 4.3)."""
    for s in (0.2, 1.6):
        p = s - math.floor(s)
        for u in UGRID[::37]:
            n, w, e = orc.assign_one(s, float(u), 10.0, hard=True)
            assert w == 1.0
            assert e == int(u > 1 - p)
            n2, w2, e2 = orc.assign_one(s, float(u), 1e12)
            assert e2 == e
            if e:
                assert abs(w2 - 1.0) < 1e-6 or abs(u - (1 - p)) < 1e-9


def test_integer_density_takes_no_extra(orc):
    for s in (1.0, 2.0, 5.0):
        for u in (0.0, 0.5, 0.999999):
            n, w, e = orc.assign_one(s, u)
            assert (n, e) == (int(s), 0)


def test_sample_count_statistics(orc):
    """E[T] = B N: the expected number of samples equals the budget (Sec. 3)."""
    rng = np.random.default_rng(11)
    d = np.exp(rng.standard_normal(1024)).astype(np.float32)
    B = 0.25
    a0 = orc.alloc(d, B, seed=1)
    p = a0.s - np.floor(a0.s)
    sigma = math.sqrt(float((p * (1 - p)).sum()))
    Ts = [orc.alloc(d, B, seed=k).T for k in range(200)]
    assert abs(np.mean(Ts) - B * d.size) < 4 * sigma / math.sqrt(len(Ts))


def test_offsets_and_sample_list(orc):
    rng = np.random.default_rng(12)
    d = np.exp(2.0 * rng.standard_normal(3000)).astype(np.float32)
    a = orc.alloc(d, 0.5)
    assert a.offsets[0] == 0 and np.all(np.diff(a.offsets) == a.counts)
    assert a.T == a.counts.sum()
    ref = np.repeat(np.arange(d.size), a.counts)
    assert np.array_equal(a.sample_pixel, ref)
    assert np.array_equal(a.counts, np.floor(a.s).astype(np.int64) + a.extra)
    assert np.all(a.w[a.extra == 0] == 1.0)


# ---------------------------------------------------------------------------
# a4: renderer stand-in (unit-mean log-normal noise, sigma = 0.8)
# ---------------------------------------------------------------------------
def test_sample_noise_distribution(orc):
    from scipy import stats
    z = np.array([orc.sample_noise(0xC0FFEE, 0, i // 4, i % 4) for i in range(40000)])
    lz = np.log(z)
    n = lz.size
    assert abs(lz.mean() + 0.32) < 5 * 0.8 / math.sqrt(n)
    assert abs(lz.std() - 0.8) < 0.02
    assert stats.kstest((lz + 0.32) / 0.8, "norm").pvalue > 1e-4
    # unit mean: E[exp(0.8 Z - 0.32)] = 1
    sd = math.sqrt(math.exp(0.64) - 1.0)
    assert abs(z.mean() - 1.0) < 5 * sd / math.sqrt(n)


# ---------------------------------------------------------------------------
# a5: splat (Eq. stoch_rnoisy) and pyramid (Eq. app-pyramid)
# ---------------------------------------------------------------------------
def test_splat_single_pixel_values(orc):
    # pixel 0: two regular samples, s = 2.0; pixel 1: one extra sample with
    # ramp weight 0.75 and s = 0.3; pixel 2: nothing
    offsets = np.array([0, 2, 3, 3], np.int64)
    rgb = np.array([[1, 2, 3], [3, 2, 1], [4, 4, 8]], np.float64)
    s = np.array([2.0, 0.3, 0.5])
    w = np.array([1.0, 0.75, 1.0])
    extra = np.array([0, 1, 0], np.int32)
    (L0,) = orc.splat(offsets, rgb, s, w, extra, 3, 1, 1)
    assert np.allclose(L0[:, 0, 0], [2.0, 2.0, 2.0], rtol=0, atol=1e-15)
    assert np.allclose(L0[:, 0, 1], np.array([4, 4, 8]) * 0.75 / 0.3, rtol=1e-15)
    assert np.all(L0[:, 0, 2] == 0.0)


@pytest.mark.parametrize("hard", [False, True])
def test_splat_unbiased(orc, hard):
    """E[L_i] = E[S_i] over the whole density range (Sec. 4.2), here with a
    unit clean image: the splatted value averages to 1."""
    W = H = 16
    N = W * H
    rng = np.random.default_rng(13)
    d = np.exp(rng.standard_normal(N)).astype(np.float32)
    clean = np.ones((3, H, W))
    acc = np.zeros(N)
    acc2 = np.zeros(N)
    K = 300
    for k in range(K):
        a = orc.alloc(d, 0.25, hard=hard, seed=k)
        rgb = orc.render(clean, a.offsets, 99, k)
        L0 = orc.splat(a.offsets, rgb, a.s, a.w, a.extra, W, H, 1)[0][0].ravel()
        acc += L0
        acc2 += L0 * L0
    mean = acc / K
    var = acc2 / K - mean**2
    # pooled z-test over all pixels
    z = (mean.mean() - 1.0) / math.sqrt(var.sum() / K) * N
    assert abs(z) < 4.5


def test_pyramid_is_block_mean(orc):
    rng = np.random.default_rng(14)
    W, H, L = 16, 8, 3
    N = W * H
    offsets = np.arange(N + 1, dtype=np.int64)
    rgb = rng.random((N, 3))
    s = np.ones(N)
    w = np.ones(N)
    extra = np.zeros(N, np.int32)
    layers = orc.splat(offsets, rgb, s, w, extra, W, H, L)
    L0 = rgb.T.reshape(3, H, W)
    assert np.allclose(layers[0], L0, rtol=0, atol=0)
    for l in range(1, L):
        b = 1 << l
        ref = L0.reshape(3, H // b, b, W // b, b).mean(axis=(2, 4))
        assert np.allclose(layers[l], ref, rtol=1e-15, atol=0)


# ---------------------------------------------------------------------------
# a6-a8: reconstruction (Appendix A)
# ---------------------------------------------------------------------------
def _rand_setup(W, H, L, seed, temporal=True):
    rng = np.random.default_rng(seed)
    layers = [rng.random((3, H >> l, W >> l)) * 4 for l in range(L)]
    logits = []
    for l in range(L):
        C = 25 if l == L - 1 else (54 if (l == 0 and temporal) else 29)
        logits.append(rng.standard_normal((C, H >> l, W >> l)))
    prev = rng.random((3, H, W)) * 4
    mv = (rng.random((2, H, W)).astype(np.float32) - 0.5) * 6
    mask = (rng.random((H, W)) < 0.2).astype(np.uint8)
    return layers, logits, prev, mv, mask


def test_constant_image_reproduced(orc):
    """Joint softmax weights sum to 1 (Eq. app-softmax-mid/full), so constant
    layers and a constant previous frame give the same constant out."""
    W, H, L = 24, 16, 3
    _, logits, _, mv, mask = _rand_setup(W, H, L, 15)
    layers = [np.full((3, H >> l, W >> l), 2.5) for l in range(L)]
    prev = np.full((3, H, W), 2.5)
    hdr, hats = orc.reconstruct(layers, logits, prev=prev, mv=mv, mask=mask)
    # G + U + temporal terms each carry part of the unit mass; levels l >= 1
    # reproduce the constant, level 0 too.
    for l in range(L):
        assert np.allclose(hats[l], 2.5, rtol=1e-14, atol=0)


def test_one_hot_centre_is_identity(orc):
    W, H, L = 16, 8, 2
    rng = np.random.default_rng(16)
    layers = [rng.random((3, H >> l, W >> l)) for l in range(L)]
    logits = []
    for l in range(L):
        C = 25 if l == L - 1 else 29
        lg = np.zeros((C, H >> l, W >> l))
        lg[12] = 60.0  # centre tap (i, j) = (0, 0)
        logits.append(lg)
    hdr, _ = orc.reconstruct(layers, logits)
    assert np.allclose(hdr, layers[0], rtol=1e-24 + 30 * math.exp(-60), atol=0)


def test_zero_logits_coarsest_is_box_filter(orc):
    """All-zero logits at the coarsest level: the 5x5 box mean with
    clamp-to-edge addressing (scipy's uniform_filter, mode='nearest')."""
    from scipy import ndimage
    rng = np.random.default_rng(17)
    img = rng.random((3, 9, 13))
    out = orc.reconstruct_level(img, np.zeros((25, 9, 13)))
    ref = np.stack([ndimage.uniform_filter(img[c], size=5, mode="nearest") for c in range(3)])
    assert np.allclose(out, ref, rtol=1e-14, atol=0)


def test_warp_zero_motion_identity_and_integer_shift(orc):
    rng = np.random.default_rng(18)
    W, H = 11, 7
    prev = rng.random((3, H, W))
    mv = np.zeros((2, H, W), np.float32)
    assert np.array_equal(orc.warp(prev, mv), prev)
    mv[0] = 2.0
    mv[1] = -1.0
    out = orc.warp(prev, mv)
    xs = np.clip(np.arange(W) + 2, 0, W - 1)
    ys = np.clip(np.arange(H) - 1, 0, H - 1)
    assert np.array_equal(out, prev[:, ys][:, :, xs])


def test_warp_bilinear_reproduces_linear_function(orc):
    """Bilinear interpolation is exact on affine images: inside the frame the
    warped value is the affine function at the displaced position."""
    W, H = 20, 12
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    a, b, c = 0.7, -0.3, 5.0
    prev = np.stack([a * xs + b * ys + c] * 3)
    rng = np.random.default_rng(19)
    mv = ((rng.random((2, H, W)) - 0.5) * 3).astype(np.float32)
    out = orc.warp(prev, mv)
    X = np.clip(xs + mv[0], 0, W - 1)
    Y = np.clip(ys + mv[1], 0, H - 1)
    assert np.allclose(out[0], a * X + b * Y + c, rtol=0, atol=1e-12)


def test_upsample_taps_as_printed(orc):
    """Eq. app-upsample: tap (i, j) reads the coarser level at
    (floor((x+i)/2), floor((y+j)/2)), clamped at the far edge."""
    Wc, Hc = 5, 3
    W, H = 2 * Wc, 2 * Hc
    rng = np.random.default_rng(20)
    coarse = rng.random((3, Hc, Wc))
    noisy = np.zeros((3, H, W))
    for (ti, tj) in [(0, 0), (1, 0), (0, 1), (1, 1)]:
        lg = np.full((29, H, W), -200.0)
        lg[25 + 2 * tj + ti] = 0.0
        out = orc.reconstruct_level(noisy, lg, coarse=coarse)
        for y in range(H):
            for x in range(W):
                xc = min((x + ti) // 2, Wc - 1)
                yc = min((y + tj) // 2, Hc - 1)
                assert abs(out[0, y, x] - coarse[0, yc, xc]) < 1e-12


def test_mask_drops_temporal_kernels(orc):
    """A disoccluded pixel's joint softmax spans only the 29 spatial logits:
    all-masked equals no temporal term at all (Sec. 6.1, Appendix A)."""
    W, H, L = 16, 8, 2
    layers, logits, prev, mv, _ = _rand_setup(W, H, L, 21)
    full = np.ones((H, W), np.uint8)
    hdr_m, _ = orc.reconstruct(layers, logits, prev=prev, mv=mv, mask=full)
    lg29 = [logits[0][:29]] + logits[1:]
    hdr_n, _ = orc.reconstruct(layers, lg29)
    assert np.allclose(hdr_m, hdr_n, rtol=1e-15, atol=0)


def _softmax(z):
    z = z - z.max(axis=0, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=0, keepdims=True)


def test_brute_force_linear_operator_8x8(orc):
    """For fixed logits the reconstruction is linear in the noisy layers and
    the warped previous frame.  Assemble it as explicit matrices from the
    definitions (G, U, W_t) and compare with the looped oracle on 8x8."""
    from scipy.special import softmax
    W = H = 8
    L = 2
    layers, logits, prev, mv, mask = _rand_setup(W, H, L, 22)
    N, Nc = W * H, (W // 2) * (H // 2)

    def gather_matrix(wt, Wl, Hl, base):
        G = np.zeros((Wl * Hl, Wl * Hl))
        for y in range(Hl):
            for x in range(Wl):
                for j in range(-2, 3):
                    for i in range(-2, 3):
                        q = min(max(y + j, 0), Hl - 1) * Wl + min(max(x + i, 0), Wl - 1)
                        G[y * Wl + x, q] += wt[base + (j + 2) * 5 + (i + 2), y, x]
        return G

    # coarsest level
    w1 = softmax(logits[1], axis=0)
    G1 = gather_matrix(w1, W // 2, H // 2, 0)
    hat1 = np.stack([G1 @ layers[1][c].ravel() for c in range(3)])
    # warp matrix: bilinear weights of every pixel
    Wt = np.zeros((N, N))
    for y in range(H):
        for x in range(W):
            X = min(max(x + float(mv[0, y, x]), 0), W - 1)
            Y = min(max(y + float(mv[1, y, x]), 0), H - 1)
            x0, y0 = int(math.floor(X)), int(math.floor(Y))
            fx, fy = X - x0, Y - y0
            x1, y1 = min(x0 + 1, W - 1), min(y0 + 1, H - 1)
            for (xx, yy, ww) in [(x0, y0, (1 - fx) * (1 - fy)), (x1, y0, fx * (1 - fy)),
                                 (x0, y1, (1 - fx) * fy), (x1, y1, fx * fy)]:
                Wt[y * W + x, yy * W + xx] += ww
    # full level: joint softmax over 54 (29 where masked)
    lg = logits[0].copy()
    lg[29:, mask.astype(bool)] = -np.inf
    w0 = softmax(lg, axis=0)
    G0 = gather_matrix(w0, W, H, 0)
    T0 = gather_matrix(w0, W, H, 29)
    U0 = np.zeros((N, Nc))
    for y in range(H):
        for x in range(W):
            for j in range(2):
                for i in range(2):
                    xc = min((x + i) // 2, W // 2 - 1)
                    yc = min((y + j) // 2, H // 2 - 1)
                    U0[y * W + x, yc * (W // 2) + xc] += w0[25 + 2 * j + i, y, x]
    ref = np.stack([G0 @ layers[0][c].ravel() + U0 @ hat1[c] + T0 @ (Wt @ prev[c].ravel())
                    for c in range(3)]).reshape(3, H, W)
    hdr, _ = orc.reconstruct(layers, logits, prev=prev, mv=mv, mask=mask)
    assert np.allclose(hdr, ref, rtol=1e-13, atol=0)


def test_reconstruction_is_linear_in_radiance(orc):
    W, H, L = 16, 16, 3
    layers, logits, prev, mv, mask = _rand_setup(W, H, L, 23)
    h1, _ = orc.reconstruct(layers, logits, prev=prev, mv=mv, mask=mask)
    h2, _ = orc.reconstruct([3.0 * x for x in layers], logits, prev=3.0 * prev, mv=mv, mask=mask)
    assert np.allclose(h2, 3.0 * h1, rtol=1e-14, atol=0)


# ---------------------------------------------------------------------------
# a9: tone map (Sec. 5)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("s,h", [(0.5, 0.5), (0.2, 0.9), (0.9, 0.2), (0.05, 0.05)])
def test_tau_c1_joins_and_bounds(orc, s, h):
    """tau is C1 at x = s-1 (value s/2, slope 1/2) and x = 1-h (value 1-h/2,
    slope 1/2); tau(0) = 1/2; 0 < dtau/dx < 1/2 off the linear segment, and
    tau in (0,1) and monotone (Sec. 5)."""
    e = 1e-7
    for x0, v0 in [(s - 1, s / 2), (1 - h, 1 - h / 2)]:
        assert abs(orc.tau(x0, s, h) - v0) < 1e-15
        assert abs(orc.tau(x0 - e, s, h) - v0 + 0.5 * e) < 1e-12
        assert abs(orc.tau(x0 + e, s, h) - v0 - 0.5 * e) < 1e-12
    assert orc.tau(0.0, s, h) == 0.5
    xs = np.linspace(-30, 30, 6001)
    t = np.array([orc.tau(float(x), s, h) for x in xs])
    assert np.all(t > 0) and np.all(t <= 1) and np.all(np.diff(t) >= 0)
    # strictly inside (0,1) wherever FP64 can tell 1 - tau from 0
    assert np.all(t[np.abs(xs) <= 1] < 1)
    dt = np.diff(t) / np.diff(xs)
    assert np.all(dt <= 0.5 + 1e-9) and np.all(dt >= 0)


def test_tau_limits_and_symmetry(orc):
    """Sec. 5's limits of the curve: at s = h = 1 no linear segment is left and
    tau(ln L) is L/2 below L = 1 and 1 - 1/(2L) above (a sigmoid in log
    radiance, symmetric about L = 1); as s, h -> 0 the toe and shoulder
    sharpen to the clamped line (1 + x)/2 on [-1, 1].  Equal shadow and
    highlight make tau point-symmetric about (0, 1/2)."""
    for L in (1e-3, 0.2, 0.5, 1.0, 2.0, 7.0, 1e3):
        t = orc.tau(math.log(L), 1.0, 1.0)
        assert abs(t - (L / 2 if L <= 1 else 1 - 1 / (2 * L))) < 1e-15
    eps = 1e-6
    for x in np.linspace(-3, 3, 121):
        t = orc.tau(float(x), eps, eps)
        assert abs(t - min(max(0.5 * (1 + x), 0.0), 1.0)) <= eps / 2 + 1e-15
    for sh in (0.1, 0.5, 0.9):
        for x in np.linspace(-4, 4, 81):
            assert abs(orc.tau(float(x), sh, sh) + orc.tau(float(-x), sh, sh) - 1) < 1e-15


def test_tonemap_derivative_bounds(orc):
    """0 < dtau/dlogL < 1/2 and 0 < dtau/dL < e/2 (Sec. 5), alpha = beta = 1."""
    Ls = np.exp(np.linspace(-12, 8, 2001))
    for s, h in [(0.5, 0.5), (0.1, 0.9), (0.95, 0.95)]:
        t = np.array([orc.tau(math.log(L), s, h) for L in Ls])
        dlog = np.diff(t) / np.diff(np.log(Ls))
        dlin = np.diff(t) / np.diff(Ls)
        assert np.all(dlog > 0) and np.all(dlog < 0.5 + 1e-9)
        assert np.all(dlin > 0) and np.all(dlin < math.e / 2)


def test_srgb_encode_inverts_iec_decode(orc):
    """IEC 61966-2-1: the encoding inverts the standard decoding
    ((V + 0.055)/1.055)^2.4 above V = 0.04045 and V/12.92 below it."""
    for V in np.linspace(0.0, 1.0, 1001):
        lin = V / 12.92 if V <= 0.04045 else ((V + 0.055) / 1.055) ** 2.4
        assert abs(orc.srgb_encode(lin) - V) < 1e-6
    assert orc.srgb_encode(0.0) == 0.0 and abs(orc.srgb_encode(1.0) - 1.0) < 1e-15


def test_tonemap_gray_and_saturation(orc):
    """A gray pixel maps every channel alike, independent of beta; L = 1 with
    k = 0 sits at tau = 1/2; beta = 0 removes all colour (Sec. 5)."""
    hdr = np.ones((3, 1, 1))
    out = orc.tonemap(hdr, 1.0, 0.3, 0.0, 0.5, 0.5)
    assert np.allclose(out, orc.srgb_encode(0.5), rtol=1e-15)
    rng = np.random.default_rng(24)
    hdr = rng.random((3, 4, 4)) * 5
    out = orc.tonemap(hdr, 1.2, 0.0, 0.3, 0.4, 0.6)
    assert np.allclose(out[0], out[1]) and np.allclose(out[1], out[2])
    # exposure: k shifts log radiance, so L e^k with k = 0 equals L with k
    a = orc.tonemap(hdr * math.exp(0.7), 1.0, 1.0, 0.0, 0.5, 0.5)
    b = orc.tonemap(hdr, 1.0, 1.0, 0.7, 0.5, 0.5)
    assert np.allclose(a, b, rtol=1e-12)


def test_oracle_results_do_not_depend_on_the_thread_count(orc):
    """The C oracle's parallel loops compute every pixel alone: one thread
    and several give the same bits."""
    import spp_inputs as inp
    W, H, L = 96, 64, 3
    x = inp.frame_inputs(W, H, L, frame=1, temporal=True)
    lg = [a.astype(np.float64) for a in x["logits"]]
    prev = np.random.default_rng(2).random((3, H, W))
    out = []
    for n in (1, 4):
        orc.set_threads(n)
        r = orc.frame(x["d"], x["clean"], lg, W, H, L, 0.5, prev=prev, mv=x["mv"],
                         mask=x["mask"], frame_index=1)
        out.append(r)
    orc.set_threads(0)
    assert np.array_equal(out[0]["alloc"].counts, out[1]["alloc"].counts)
    assert np.array_equal(out[0]["rgb"], out[1]["rgb"])
    assert np.array_equal(out[0]["hdr"], out[1]["hdr"])
    assert np.array_equal(out[0]["ldr"], out[1]["ldr"])
