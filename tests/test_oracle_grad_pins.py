"""Pins of the oracle's analytic gradients (a11) against central finite
differences of the oracle's own forward functions, in FP64.

Each backward function is the chain rule written out by hand; a dropped
term, a wrong sign or a transposed index shows up as a mismatch with the
finite difference of the forward.  Sizes are small (8 x 8 .. 16 x 12) so the
whole file runs in seconds.
"""
import math

import numpy as np
import pytest

EPS = 1e-6


def _fd(f, x, idx, eps=EPS):
    xp = x.copy()
    xm = x.copy()
    xp.flat[idx] += eps
    xm.flat[idx] -= eps
    return (f(xp) - f(xm)) / (2 * eps)


def _check(f, x, grad, rng, n=40, rtol=1e-5, atol=2e-8):
    for idx in rng.choice(x.size, size=min(n, x.size), replace=False):
        fd = _fd(f, x, int(idx))
        assert abs(fd - grad.flat[idx]) <= rtol * max(abs(fd), abs(grad.flat[idx])) + atol, \
            (int(idx), fd, grad.flat[idx])


@pytest.mark.parametrize("variant", ["coarsest", "mid", "full", "full_masked"])
def test_reconstruct_level_backward_matches_fd(orc, variant):
    """App. A: gradients of sum(g * out) with respect to the logits (through
    the joint softmax), the noisy level, the coarser level and the warped
    previous frame (through G, U and the temporal gather)."""
    rng = np.random.default_rng(100)
    W, H = 12, 8
    noisy = rng.random((3, H, W)) * 2
    g = rng.standard_normal((3, H, W))
    coarse = warped = mask = None
    C = 25
    if variant != "coarsest":
        coarse = rng.random((3, H // 2, W // 2)) * 2
        C = 29
    if variant.startswith("full"):
        warped = rng.random((3, H, W)) * 2
        C = 54
        if variant == "full_masked":
            mask = (rng.random((H, W)) < 0.3).astype(np.uint8)
    logits = rng.standard_normal((C, H, W)) * 1.5

    def loss(lg=logits, nz=noisy, cs=coarse, wp=warped):
        return float((orc.reconstruct_level(nz, lg, coarse=cs, warped=wp, mask=mask) * g).sum())

    gl, gn, gc, gw = orc.reconstruct_level_backward(noisy, logits, g, coarse=coarse, warped=warped,
                                                    mask=mask)
    _check(lambda x: loss(lg=x), logits, gl, rng)
    _check(lambda x: loss(nz=x), noisy, gn, rng)
    if coarse is not None:
        _check(lambda x: loss(cs=x), coarse, gc, rng)
    if warped is not None:
        _check(lambda x: loss(wp=x), warped, gw, rng)
    if mask is not None:  # disoccluded pixels have no temporal gradient
        assert np.all(gl[29:, mask.astype(bool)] == 0.0)
    # softmax invariance: the logit gradient of each pixel sums to zero
    assert np.allclose(gl.sum(axis=0), 0.0, atol=1e-12)


def test_warp_backward_matches_fd(orc):
    rng = np.random.default_rng(101)
    W, H = 10, 7
    prev = rng.random((3, H, W))
    mv = ((rng.random((2, H, W)) - 0.5) * 5).astype(np.float32)
    g = rng.standard_normal((3, H, W))
    gp = orc.warp_backward(mv, g)
    _check(lambda x: float((orc.warp(x, mv) * g).sum()), prev, gp, rng)
    # the warp is linear: sum over the image of g * W(prev) equals <W^T g, prev>
    assert abs(float((orc.warp(prev, mv) * g).sum()) - float((gp * prev).sum())) < 1e-12


@pytest.mark.parametrize("tm", [(1.0, 1.0, 0.0, 0.5, 0.5), (1.2, 0.7, -0.4, 0.3, 0.8)])
def test_tonemap_backward_matches_fd(orc, tm):
    """Sec. 5: gradient through sRGB, tau, contrast, saturation, exposure
    and the log of the radiance."""
    rng = np.random.default_rng(102)
    hdr = np.exp(rng.standard_normal((3, 6, 5)) * 2)
    gl = rng.standard_normal(hdr.shape)
    gh = orc.tonemap_backward(hdr, gl, *tm)
    _check(lambda x: float((orc.tonemap(x, *tm) * gl).sum()), hdr, gh, rng)


def test_l1_loss_gradient(orc):
    rng = np.random.default_rng(103)
    a = rng.random(50)
    b = rng.random(50)
    v, g = orc.l1_loss(a, b)
    assert abs(v - np.abs(a - b).mean()) < 1e-15
    _check(lambda x: orc.l1_loss(x, b)[0], a, g, rng)


def test_pyramid_backward_is_transpose_of_pooling(orc):
    """Eq. app-pyramid is linear; its backward is the transposed operator:
    <pool(x), g> = <x, pool^T(g)> for every level."""
    rng = np.random.default_rng(104)
    W, H, L = 16, 8, 3
    N = W * H
    offsets = np.arange(N + 1, dtype=np.int64)
    x = rng.random((N, 3))
    layers = orc.splat(offsets, x, np.ones(N), np.ones(N), np.zeros(N, np.int32), W, H, L)
    gls = [rng.standard_normal((3, H >> l, W >> l)) for l in range(L)]
    g0 = orc.pyramid_backward(gls, W, H)
    lhs = sum(float((layers[l] * gls[l]).sum()) for l in range(L))
    rhs = float((x.T.reshape(3, H, W) * g0).sum())
    assert abs(lhs - rhs) < 1e-12


def test_splat_backward_matches_fd(orc):
    """Eq. stoch_rnoisy with the ramp of Eq. relaxed_holdout: dL0/ds through
    the 1/s normalisation and the ramp weight (discrete decisions held fixed,
    as they are between thresholds)."""
    rng = np.random.default_rng(105)
    W, H = 16, 8
    N = W * H
    d = np.exp(rng.standard_normal(N)).astype(np.float32)
    seed, frame, lam = 77, 3, 10.0
    a = orc.alloc(d, 0.6, lam=lam, seed=seed, frame=frame)
    rgb = rng.random((a.T, 3)) + 0.1
    u = np.array([orc.pixel_uniform(seed, frame, i) for i in range(N)])
    g = rng.standard_normal((3, H, W))

    def L0_of(s_vec):
        w = np.array([orc.assign_one(float(s_vec[i]), float(u[i]), lam)[1] for i in range(N)])
        return orc.splat(a.offsets, rgb, s_vec, w, a.extra, W, H, 1)[0]

    L0 = L0_of(a.s)
    gs = orc.splat_backward(a, rgb, L0, g, lam=lam, seed=seed, frame=frame)
    checked = 0
    for i in range(N):
        p = a.s[i] - math.floor(a.s[i])
        if min(p, 1 - p) < 1e-4:
            continue  # next to an integer the count itself changes
        if a.extra[i]:
            r = lam / p * (u[i] + p - 1)
            if min(abs(r), abs(r - 1)) < 1e-3:
                continue  # at a corner of the ramp
        fd = _fd(lambda s: float((L0_of(s) * g).sum()), a.s, i, eps=1e-6)
        assert abs(fd - gs[i]) <= 1e-5 * max(abs(fd), abs(gs[i])) + 1e-8, (i, fd, gs[i])
        checked += 1
    assert checked > N // 2
    # some pixels are on the ramp's linear region, so that term is exercised
    lin = [(a.extra[i] and 0 < lam / (a.s[i] % 1) * (u[i] + a.s[i] % 1 - 1) < 1) for i in range(N)]
    assert any(lin)


def test_density_backward_matches_fd(orc):
    """Sec. 3: gradient of s = phi B + (1 - phi) B N softmax(z) with respect
    to the sampler logits z; it sums to zero (softmax invariance)."""
    rng = np.random.default_rng(106)
    z = rng.standard_normal(64)
    g = rng.standard_normal(64)
    B = 0.25
    gz = orc.density_backward(z, g, B)
    _check(lambda x: float((orc.density_forward(x, B) * g).sum()), z, gz, rng, n=64)
    assert abs(gz.sum()) < 1e-12
    # the FP64 forward agrees with the production definition on exp(z)
    s = orc.density_forward(z, B)
    a = orc.alloc(np.exp(z - z.max()).astype(np.float32), B)
    assert abs(s.sum() - B * 64) < 1e-12
    assert np.allclose(s, a.s, rtol=1e-6)
