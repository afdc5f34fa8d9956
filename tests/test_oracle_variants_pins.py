"""Pins of the variant oracles (oracle/variants.py) against closed forms,
a library reshape-mean and finite differences."""
import numpy as np
import pytest

import oracle
import oracle.variants as V


def _p64(d, W, H, f):
    m = np.asarray(d, np.float64).reshape(H // f, f, W // f, f).mean(axis=(1, 3))
    return np.repeat(np.repeat(m, f, axis=0), f, axis=1).reshape(-1)


@pytest.mark.parametrize("f", [2, 4])
def test_density_lowres_is_the_block_mean(f):
    W, H = 24, 16
    d = np.random.default_rng(f).lognormal(size=H * W).astype(np.float32)
    got = V.density_lowres(d, W, H, f)
    assert got.dtype == np.float32
    assert np.allclose(got, _p64(d, W, H, f), rtol=1e-6, atol=0)
    # block-constant images are fixed points (bit for bit), the sum is kept
    assert np.array_equal(V.density_lowres(got, W, H, f), got)
    assert abs(got.astype(np.float64).sum() - d.astype(np.float64).sum()) < 1e-5 * d.sum()
    # symmetry <P a, b> = <a, P b> (FP64 projection)
    b = np.random.default_rng(7).standard_normal(H * W)
    assert abs(_p64(d, W, H, f) @ b - d.astype(np.float64) @ _p64(b, W, H, f)) < 1e-9 * np.abs(b).sum()


def test_density_gradient_through_the_projection(orc):
    """s = phi B + (1 - phi) B N (P d) / sum d with d = exp(z - max z): since
    P is symmetric and keeps the sum, dLoss/dz is the density backward of
    P applied to dLoss/ds (Sec. 3 normalisation); checked by central FD."""
    W, H, f, B, phi = 8, 8, 2, 0.25, 0.125
    rng = np.random.default_rng(3)
    z = rng.standard_normal(H * W)
    g = rng.standard_normal(H * W)

    def loss(zz):
        d = np.exp(zz - zz.max())
        s = B * phi + (1 - phi) * B * (H * W) * _p64(d, W, H, f) / d.sum()
        return float(g @ s)

    gz = orc.density_backward(z, _p64(g, W, H, f), B, phi)
    for i in range(0, H * W, 5):
        zp, zm = z.copy(), z.copy()
        zp[i] += 1e-6
        zm[i] -= 1e-6
        fd = (loss(zp) - loss(zm)) / 2e-6
        assert abs(fd - gz[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gz[i])


# ------------------------------------------------------ systematic rounding
@pytest.mark.parametrize("B,seed", [(0.25, 1), (0.125, 2), (1.7, 3)])
def test_systematic_total_is_the_budget(orc, B, seed):
    """T = floor((sum q + U) / 2^32) is within one sample of B N (the q_i
    round s_i to 2^-33, and sum s_i = B N up to FP64 rounding)."""
    W, H = 64, 48
    d = np.random.default_rng(seed).lognormal(sigma=1.5, size=W * H).astype(np.float32)
    a = V.alloc_systematic(d, B, seed=seed, frame=4)
    assert a.T == (int(a.q.sum()) + a.U) >> 32
    assert abs(a.T - B * W * H) < 1 + W * H * 2.0 ** -32
    f = a.q >> 32
    assert np.all((a.counts == f) | (a.counts == f + 1))
    assert a.offsets[0] == 0 and np.all(np.diff(a.offsets) >= 0)


def test_systematic_is_unbiased_over_the_offset(orc):
    """Over all frame offsets U on the 2^-12 grid, the mean count of every
    pixel is q_i 2^-32 to within 2^-12 (its interval covers q_i 2^-32
    integers on average)."""
    d = np.random.default_rng(5).lognormal(size=12).astype(np.float32)
    counts = np.zeros(12)
    K = 1 << 12
    for k in range(K):
        counts += V.alloc_systematic(d, 0.4, U=k << 20).counts
    mean = counts / K
    assert np.all(np.abs(mean - V.alloc_systematic(d, 0.4, U=0).q * 2.0 ** -32) <= 2.0 ** -12 + 1e-12)


def test_systematic_constant_density_is_evenly_spaced(orc):
    W, H = 32, 8
    d = np.ones(W * H, np.float32)
    a = V.alloc_systematic(d, 0.25, seed=9)
    idx = np.flatnonzero(a.counts)
    assert a.T == 64 and np.all(np.diff(idx) == 4)  # every 4th pixel


def test_systematic_decision_is_the_stochastic_rule_at_u_a(orc):
    """The C oracle's stochastic assignment (Sec. 4.2-4.3), given s = q 2^-32
    and u = a_i, returns the same counts and ramp weights."""
    W, H = 40, 20
    d = np.random.default_rng(6).lognormal(size=W * H).astype(np.float32)
    a = V.alloc_systematic(d, 0.6, seed=3, frame=2)
    for i in range(W * H):
        s = float(a.q[i]) * 2.0 ** -32
        u = float(a.a32[i]) * 2.0 ** -32
        if abs(u - (1.0 - (s - np.floor(s)))) < 1e-12:
            continue  # the tie a + p = 1 (the ramp is 0 there either way)
        n, w, e = orc.assign_one(s, u, 10.0, False)
        assert n == a.counts[i], i
        if e:
            assert abs(w - float(a.w[i])) <= 1e-6 * max(1.0, abs(w)), i


# ------------------------------------------------ gradient estimators
def _gumbel_case(orc, W=12, H=8, B=0.6, lam=4.0):
    d = np.random.default_rng(21).lognormal(size=W * H).astype(np.float32)
    a = V.alloc_gumbel(d, B, lam=lam, seed=31, frame=2)
    clean, _ = __import__("spp_inputs").scene(W, H, seed=5)
    rgb = orc.render(clean, a.offsets, 0xC0FFEE, 2)
    return a, rgb, clean, W, H


def test_gumbel_gradient_matches_fd(orc):
    """With u and the traced set fixed, L^0 is a smooth function of s: the
    estimator's gradient is its exact derivative."""
    lam = 4.0
    a, rgb, clean, W, H = _gumbel_case(orc, lam=lam)
    g = np.random.default_rng(22).standard_normal((3, H * W))
    f = np.floor(a.s)

    def L0_of(s):
        w = np.where(a.extra, V.gumbel_weight(np.where(a.extra, s - f, 0.5), a.u, lam), 1.0)
        return orc.splat(a.offsets, rgb, s, w, a.extra, W, H, 1)[0].reshape(3, -1)

    L0 = L0_of(a.s)
    grad = V.splat_backward_estimator(a, rgb, L0, g, "gumbel", lam=lam)
    for i in np.flatnonzero(a.extra)[:25]:
        if not (1e-4 < a.p[i] < 1 - 1e-4):
            continue
        sp, sm = a.s.copy(), a.s.copy()
        sp[i] += 1e-7
        sm[i] -= 1e-7
        fd = float((g * (L0_of(sp) - L0_of(sm))).sum()) / 2e-7
        assert abs(fd - grad[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, grad[i])


def test_gumbel_hard_limit_is_the_stochastic_rule(orc):
    """As lambda grows, w -> [u > 1 - p]: the test-time decision of the
    Gumbel estimator is the stochastic map of Sec. 4.2."""
    W, H = 16, 16
    d = np.random.default_rng(23).lognormal(size=W * H).astype(np.float32)
    a = V.alloc_gumbel(d, 0.4, lam=1e9, seed=7, frame=1)
    ref = orc.alloc(d, 0.4, hard=True, seed=7, frame=1)
    hard_extra = a.extra & (a.w > 0.5)
    assert np.array_equal(np.floor(a.s).astype(np.int64) + hard_extra, ref.counts)


def test_straight_through_uses_the_renderers_sample(orc):
    """The untraced sample of slot f is the renderer stand-in's sample of
    that slot (the one it returns when the pixel gets f + 1 samples), and
    dLoss/ds = sum_c g_c (S_f,c - L^0_c) / s on a pixel with p > 0."""
    W, H = 6, 4
    d = np.random.default_rng(24).lognormal(size=W * H).astype(np.float32)
    a = orc.alloc(d, 0.7, hard=True, seed=9, frame=3)
    clean, _ = __import__("spp_inputs").scene(W, H, seed=6)
    rgb = orc.render(clean, a.offsets, 0xBEEF, 3)
    L0 = orc.splat(a.offsets, rgb, a.s, a.w, a.extra, W, H, 1)[0].reshape(3, -1)
    g = np.random.default_rng(25).standard_normal((3, H * W))
    grad = V.splat_backward_estimator(a, rgb, L0, g, "straight_through", clean=clean,
                                      render_seed=0xBEEF, frame=3)
    i = int(np.flatnonzero((a.counts == np.floor(a.s)) & (a.s > np.floor(a.s)))[0])
    more = a.counts.copy()
    more[i] += 1  # the same frame with one more sample on pixel i
    off2 = np.concatenate([[0], np.cumsum(more)])
    S_f = orc.render(clean, off2, 0xBEEF, 3)[off2[i + 1] - 1]
    expect = float(g[:, i] @ (S_f - L0[:, i])) / a.s[i]
    assert abs(grad[i] - expect) <= 1e-12 * max(1.0, abs(expect))


# ------------------------------------------------ DASR (Sec. 4.1, Eq. kuz_fw / kuz_grad)
def test_dasr_counts_at_and_around_the_half_integers():
    """round(s) of Eq. kuz_fw by hand: halves go up, so s >= 1/2 gives at
    least one sample and s < 1/2 none."""
    below = lambda x: np.nextafter(x, 0.0)  # noqa: E731
    s = [0.0, 1e-300, 0.25, below(0.5), 0.5, 0.51, 1.0, 1.49, below(1.5), 1.5, 2.5, 3.0,
         7.49, 7.5]
    want = [0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 3, 3, 7, 8]
    assert V.dasr_counts(s).tolist() == want


def test_dasr_counts_are_the_nearest_integer_exactly():
    """|n - s| <= 1/2 in exact rational arithmetic, and a tie goes up."""
    from fractions import Fraction
    rng = np.random.default_rng(12)
    s = np.concatenate([rng.lognormal(-1.0, 1.5, 2000), np.arange(0, 40) * 0.5,
                        np.nextafter(np.arange(1, 40) * 0.5, 0.0)])
    for si, ni in zip(s, V.dasr_counts(s)):
        e = Fraction(int(ni)) - Fraction(float(si))
        assert abs(e) <= Fraction(1, 2)
        if abs(e) == Fraction(1, 2):
            assert e > 0


def test_dasr_forward_is_the_sample_mean_and_zero_without_samples():
    """Eq. kuz_fw on a 2 x 2 frame by hand, and the level-1 block mean."""
    counts = [0, 1, 3, 2]
    rgb = [(1, 2, 3),                                   # pixel 1
           (1, 0, 0), (2, 0, 0), (6, 3, 0),             # pixel 2
           (4, 4, 4), (0, 2, 8)]                        # pixel 3
    l0, l1 = V.splat_dasr(counts, rgb, 2, 2, 2)
    want = np.array([[0, 0, 0], [1, 2, 3], [3, 1, 0], [2, 3, 6]], np.float64).T.reshape(3, 2, 2)
    assert np.array_equal(l0, want)
    assert np.allclose(l1.ravel(), [1.5, 1.5, 2.25], rtol=0, atol=1e-15)


def test_dasr_alloc_budget_and_threshold():
    """round() moves each pixel by at most 1/2, so the total is within N/2
    of B N (Sec. 3 fixes sum s = B N); a pixel is sampled iff s >= 1/2."""
    W, H, B = 64, 48, 0.75
    d = np.random.default_rng(4).lognormal(size=W * H).astype(np.float32)
    a = V.alloc_dasr(d, B)
    assert np.array_equal(a.counts, V.dasr_counts(a.s))
    assert abs(a.T - B * W * H) <= W * H / 2
    assert np.array_equal(a.counts >= 1, a.s >= 0.5)
    assert np.array_equal(np.diff(a.offsets), a.counts)
    assert np.array_equal(a.norm, np.maximum(a.counts, 1))
    # a uniform density puts s = B on every pixel (exact here): B = 2.5 rounds up
    u = V.alloc_dasr(np.ones(256, np.float32), 2.5)
    assert np.all(u.s == 2.5) and np.all(u.counts == 3) and u.T == 768


def test_dasr_surrogate_gradient_by_hand():
    """Eq. kuz_grad: (L^ref - L^0) / round(s) where sampled, L^ref where not,
    each dotted with the loss gradient of the pixel's three channels."""
    counts = [2, 0]
    L0 = np.array([[3, 3, 3], [0, 0, 0]], np.float64).T
    ref = np.array([[2, 2, 2], [1, 2, 3]], np.float64).T
    g = np.array([[1, 0, 2], [1, 1, 1]], np.float64).T
    got = V.splat_backward_dasr(counts, L0, g, ref)
    assert got.tolist() == [(1 * -1 + 0 + 2 * -1) / 2, 1 + 2 + 3]
