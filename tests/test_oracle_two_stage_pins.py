"""Pins of the two-stage pipeline oracle (oracle/two_stage.py, the network
specifications of oracle/unet.py) against things other than the code under
test: the splat oracle's own pyramid, the plain reconstruction, the exact
cancellation of a constant demodulation map, central finite differences and
closed forms of the parameter counts and feature channels."""
import math

import numpy as np
import pytest

import oracle.two_stage as TS
import oracle.unet as U
import spp_inputs as inp


def _fd_check(f, x, grad, rng, n=30, eps=1e-6, rtol=1e-5, atol=1e-8):
    for idx in rng.choice(x.size, size=min(n, x.size), replace=False):
        xp, xm = x.copy(), x.copy()
        xp.flat[idx] += eps
        xm.flat[idx] -= eps
        fd = (f(xp) - f(xm)) / (2 * eps)
        g = grad.flat[idx]
        assert abs(fd - g) <= rtol * max(abs(fd), abs(g)) + atol, (int(idx), fd, g)


def test_param_counts_closed_form():
    def count(cin, heads):
        c0, c1, c2 = heads
        convs = [(cin, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (192, 64),
                 (64, 64), (96, 32), (32, 32), (32, c0)]
        if c1:
            convs.append((64, c1))
        if c2:
            convs.append((128, c2))
        return sum(9 * a * b + b for a, b in convs)
    assert U.param_offsets("joint")[1] == count(12, (55, 29, 25)) == 535565
    assert U.param_offsets("sampler")[1] == count(19, (1, 0, 0))
    assert U.param_offsets("denoiser")[1] == count(24, (64, 29, 25))
    assert [n for n, *_ in U.layers("sampler")] == ["e0a", "e0b", "e1a", "e1b", "e2a", "e2b",
                                                     "d1a", "d1b", "d0a", "d0b", "h0"]


def test_pyramid_equals_the_splat_pyramid(orc):
    """Eq. app-pyramid as built by the splat oracle (C, from the samples)
    and by block means of its level 0 agree."""
    W, H = 32, 16
    d = inp.density_lognormal(W, H, seed=3)
    clean, _ = inp.scene(W, H, seed=4)
    a = orc.alloc(d, 0.5, seed=11, frame=0)
    rgb = orc.render(clean, a.offsets, 0xC0FFEE, 0)
    layers = orc.splat(a.offsets, rgb, a.s, a.w, a.extra, W, H, 3)
    pyr = TS.pyramid(layers[0], 3)
    for l in (1, 2):
        assert np.allclose(pyr[l], layers[l], rtol=1e-13, atol=1e-300)


def _frame_inputs(W, H, L, seed, temporal=True):
    rng = np.random.default_rng(seed)
    L0 = rng.random((3, H, W)) * 3
    logits = [z.astype(np.float64) for z in inp.random_logits(W, H, L, seed=seed, temporal=temporal)]
    warped = rng.random((3, H, W)) * 2 if temporal else None
    mask = (rng.random((H, W)) < 0.2).astype(np.uint8) if temporal else None
    return L0, logits, warped, mask


@pytest.mark.parametrize("temporal", [False, True])
def test_unit_demodulation_is_the_plain_reconstruction(orc, temporal):
    W, H, L = 16, 8, 3
    L0, logits, warped, mask = _frame_inputs(W, H, L, 5, temporal)
    hdr, _ = TS.reconstruct_demod(L0, np.zeros((3, H, W)), logits, warped, mask, L)
    layers = TS.pyramid(L0, L)
    ref = None
    for l in range(L - 1, -1, -1):
        ref = orc.reconstruct_level(layers[l], logits[l], ref, warped if l == 0 else None,
                                    mask if l == 0 else None)
    assert np.array_equal(hdr, ref)


def test_constant_demodulation_cancels(orc):
    """Sec. 6.2: the gathers are linear in the radiance and their weights do
    not depend on it, so a per-channel constant m divides out exactly."""
    W, H, L = 16, 8, 3
    L0, logits, warped, mask = _frame_inputs(W, H, L, 6)
    c = np.broadcast_to(np.array([0.7, -1.3, 2.9])[:, None, None], (3, H, W)).copy()
    hdr, _ = TS.reconstruct_demod(L0, c, logits, warped, mask, L)
    ref, _ = TS.reconstruct_demod(L0, np.zeros((3, H, W)), logits, warped, mask, L)
    assert np.allclose(hdr, ref, rtol=1e-13, atol=0)
    # a spatially varying map does change the result
    c2 = c + np.random.default_rng(1).standard_normal((3, H, W))
    hdr2, _ = TS.reconstruct_demod(L0, c2, logits, warped, mask, L)
    assert np.abs(hdr2 - ref).max() > 1e-3


@pytest.mark.parametrize("temporal", [False, True])
def test_demod_backward_matches_fd(orc, temporal):
    W, H, L = 8, 8, 2
    L0, logits, warped, mask = _frame_inputs(W, H, L, 7, temporal)
    rng = np.random.default_rng(8)
    c = rng.uniform(-2, 2, (3, H, W))
    g = rng.standard_normal((3, H, W))
    g_logits, g_L0, g_c = TS.reconstruct_demod_backward(L0, c, logits, g, warped, mask, L)
    loss = lambda L0_, c_, lg: float((g * TS.reconstruct_demod(L0_, c_, lg, warped, mask, L)[0]).sum())
    _fd_check(lambda x: loss(x, c, logits), L0, g_L0, rng)
    _fd_check(lambda x: loss(L0, x, logits), c, g_c, rng)
    # outside the clamp m does not move: the gradient is exactly zero there
    cc = c.copy()
    cc[0, 0, :3] = [9.0, -9.5, 8.5]
    _, _, g_cc = TS.reconstruct_demod_backward(L0, cc, logits, g, warped, mask, L)
    assert np.all(g_cc[0, 0, :3] == 0) and np.all(g_cc[1:] != 0)
    for l in range(L):
        def f(x, l=l):
            lg = list(logits)
            lg[l] = x
            return loss(L0, c, lg)
        _fd_check(f, logits[l], g_logits[l], rng, n=20)


@pytest.mark.parametrize("spec", ["sampler", "denoiser"])
def test_network_input_and_parameter_gradients_match_fd(spec):
    cin, heads = U.SPECS[spec]
    table, total = U.param_offsets(spec)
    rng = np.random.default_rng(9)
    theta = inp.unet_params(U.layers(spec), seed=10).astype(np.float64)
    for name, ci, co, wo, bo in table:
        theta[bo:bo + co] = 0.1 * rng.standard_normal(co)
    H = W = 8
    x = rng.standard_normal((cin, H, W))
    gh = [None if c == 0 else rng.standard_normal((c, H >> l, W >> l))
          for l, c in enumerate(heads)]
    fwd = U.forward(theta, x, spec=spec)
    g_theta, g_x = U.backward_heads(fwd, gh, input_grad=True)

    def loss(th, xx):
        hs = U.forward(th, xx, spec=spec)["heads"]
        return float(sum((a * b).sum() for a, b in zip(hs, gh) if b is not None))
    _fd_check(lambda xx: loss(theta, xx), x, g_x, rng, n=25, rtol=1e-5, atol=1e-7)
    _fd_check(lambda th: loss(th, x), theta, g_theta, rng, n=25, rtol=1e-5, atol=1e-7)


def test_feature_channel_layout():
    H, W = 4, 8
    rng = np.random.default_rng(12)
    L0 = rng.random((3, H, W))
    s = rng.random(H * W) + 0.1
    n = rng.integers(0, 3, H * W)
    alb, nrm = rng.random((3, H, W)), rng.standard_normal((3, H, W))
    depth = rng.uniform(1, 100, (H, W))
    mv = rng.uniform(-8, 8, (2, H, W))
    prev = rng.random((3, H, W))
    lat = rng.uniform(-1, 1, (TS.N_LATENT, H, W))
    x = TS.denoiser_features(L0, s, n, alb, nrm, depth, mv, prev, lat)
    assert x.shape == (24, H, W) and U.SPECS["denoiser"][0] == 24
    assert np.allclose(np.expm1(x[0:3]), L0, rtol=1e-14)
    assert np.allclose(np.expm1(x[3]).ravel(), s) and np.allclose(np.expm1(x[4]).ravel(), n)
    assert np.array_equal(x[5:8], alb) and np.array_equal(x[8:11], nrm)
    assert np.allclose(100.0 ** x[11], depth)
    assert np.allclose(8 * x[12:14], mv)
    assert np.allclose(np.expm1(x[14:17]), prev) and np.array_equal(x[17:24], lat)
    y = TS.sampler_features(alb, nrm, depth, mv, prev, lat)
    assert y.shape == (19, H, W) and U.SPECS["sampler"][0] == 19
    assert np.array_equal(y[9:12], prev) and np.array_equal(y[12:19], lat)
    g_x = rng.standard_normal((24, H, W))
    g_L0, g_s = TS.denoiser_features_backward(L0, s, g_x)
    # d ln(1 + v) / dv = 1 / (1 + v)
    assert np.allclose(g_L0, g_x[0:3] / (1 + L0)) and np.allclose(g_s.ravel(), g_x[3].ravel() / (1 + s))


def test_demod_map_and_latents():
    h0 = np.zeros((64, 2, 2))
    h0[54:57] = np.array([0.0, 9.0, -20.0])[:, None, None]
    h0[57:64] = 0.5
    m = TS.demod_map(h0)
    assert np.all(m[0] == 1.0) and np.allclose(m[1], math.exp(8.0)) and np.allclose(m[2], math.exp(-8.0))
    assert np.allclose(TS.latent(h0), math.tanh(0.5))


def test_warp_channels_matches_the_frame_warp(orc):
    W, H = 12, 8
    rng = np.random.default_rng(13)
    f = rng.random((7, H, W))
    mv = inp.motion_affine(W, H, seed=2)
    out = TS.warp_channels(f, mv)
    for k in range(7):
        ref = orc.warp(np.stack([f[k]] * 3), mv)[0]
        assert np.array_equal(out[k], ref)
