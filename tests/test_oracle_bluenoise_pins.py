"""Pins of the blue-noise dither oracle (oracle/bluenoise.py): the mask is
a permutation with blue-noise structure (low frequencies suppressed, points
spread out), the uniforms are exactly stratified per tile, and a constant
density receives its budget to within one sample per tile."""
import numpy as np
import pytest

import oracle
import oracle.bluenoise as BN


@pytest.fixture(scope="module")
def m64():
    return BN.mask(64, seed=7)


def test_weights_are_a_toroidal_gaussian():
    w = BN.weights(32)
    assert w[0, 0] == 2 ** 20
    assert np.array_equal(w, w.T) and np.array_equal(w[1:], w[1:][::-1])
    r2 = np.minimum(np.arange(32), 32 - np.arange(32)) ** 2
    d2 = r2[:, None] + r2[None, :]
    order = np.argsort(d2.ravel(), kind="stable")
    assert np.all(np.diff(w.ravel()[order]) <= 0)  # non-increasing with distance
    assert abs(w[0, 1] / 2 ** 20 - np.exp(-1 / 4.5)) < 1e-6


def test_mask_is_a_permutation(m64):
    assert m64.shape == (64, 64)
    assert np.array_equal(np.sort(m64.ravel()), np.arange(4096))


def _low_freq_power(binary):
    F = np.abs(np.fft.fft2(binary - binary.mean())) ** 2
    f = np.fft.fftfreq(binary.shape[0]) * binary.shape[0]
    rad = np.sqrt(f[:, None] ** 2 + f[None, :] ** 2)
    return F[(rad > 0) & (rad <= binary.shape[0] / 8)].mean()


@pytest.mark.parametrize("level", [0.1, 0.25, 0.5, 0.75])
def test_threshold_patterns_are_blue(m64, level):
    """Every threshold level of a blue-noise mask is a pattern whose power
    spectrum is suppressed at low frequencies (Ulichney's definition); a
    random permutation (white noise) is the comparison."""
    rng = np.random.default_rng(1)
    white = rng.permutation(4096).reshape(64, 64)
    k = int(level * 4096)
    blue = (m64 < k).astype(float)
    wn = (white < k).astype(float)
    assert _low_freq_power(blue) < 0.1 * _low_freq_power(wn)


def test_sparse_levels_keep_points_apart(m64):
    """The 1 % level (41 points on 64 x 64) has a nearest-neighbour distance
    well above that of white noise of the same density."""
    pts = np.argwhere(m64 < 41)
    d = np.abs(pts[:, None, :] - pts[None, :, :])
    d = np.minimum(d, 64 - d)
    dist = np.sqrt((d ** 2).sum(-1)) + np.eye(len(pts)) * 1e9
    assert dist.min() >= 5.0


def test_mask_depends_on_seed_only():
    a, b = BN.mask(16, 3), BN.mask(16, 3)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, BN.mask(16, 4))


def test_uniforms_are_stratified_per_tile(m64):
    """Within one tile and frame the uniforms are the T^2 stratified values
    (r + 1/2) / T^2 shifted by one offset; the next frame adds G48."""
    u0 = BN.uniform48(m64, 64, 64, seed=5, frame=0).astype(object)
    u1 = BN.uniform48(m64, 64, 64, seed=5, frame=1).astype(object)
    off = (u0[0] - (int(m64[0, 0]) << 36) - (1 << 35)) % (1 << 48)
    base = sorted((v - off) % (1 << 48) for v in u0)
    assert base == [(r << 36) + (1 << 35) for r in range(4096)]
    assert all((b - a) % (1 << 48) == BN.G48 for a, b in zip(u0, u1))


def test_constant_density_gets_its_budget_per_tile(m64):
    """With d constant every pixel has s = B; over one T x T tile the number
    of extra samples is the number of stratified uniforms above 1 - p, so T
    differs from B N by at most one sample per tile (white noise: about
    sqrt(B N (1-p)))."""
    orc = oracle
    orc.build()
    W = H = 128
    d = np.ones(W * H, np.float32)
    for B, frame in [(0.25, 0), (0.37, 3), (1.6, 5)]:
        u = BN.uniform48(m64, W, H, seed=9, frame=frame)
        a = orc.alloc(d, B, u48=u)
        assert abs(a.T - B * W * H) <= 4  # 4 tiles
