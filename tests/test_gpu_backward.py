"""Parity of the CUDA backward kernels (a11) with the oracle's analytic
gradients, which tests/test_oracle_grad_pins.py pins to FP64 finite
differences.

Tolerance: |gpu - oracle| <= 1e-4 |oracle| + 1e-5 max|oracle| per element.
The relative part is the FP32 target; the small absolute part covers
gradients that are differences of nearly equal terms (the softmax gradient
w_k (q_k - sum_j w_j q_j), the splat's two terms), whose relative error is
not bounded by the inputs'.
"""
import numpy as np
import pytest
import torch

import oracle
import spp_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spp():
    from conftest import build_spp_lib
    build_spp_lib()
    import paper_2602_08642_gb300 as spp
    torch.cuda.set_device(0)
    return spp


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def assert_grad(got, ref, what, rtol=1e-4, afrac=1e-5):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape, what
    bound = rtol * np.abs(ref) + afrac * max(float(np.abs(ref).max()), 1e-30)
    bad = np.abs(got - ref) > bound
    if bad.any():
        k = int(np.argmax(np.abs(got - ref) / bound))
        raise AssertionError(f"{what}: {int(bad.sum())} out of tolerance; worst flat {k}: "
                             f"got {got.ravel()[k]!r} ref {ref.ravel()[k]!r}")


def _level_inputs(W, H, variant, seed):
    rng = np.random.default_rng(seed)
    noisy = (rng.random((3, H, W)) * 2).astype(np.float32)
    noisy[:, rng.random((H, W)) < 0.5] = 0.0
    g = rng.standard_normal((3, H, W)).astype(np.float32)
    coarse = warped = mask = None
    C = 25
    if variant != "coarsest":
        coarse = (rng.random((3, H // 2, W // 2)) * 2).astype(np.float32)
        C = 29
    if variant.startswith("full"):
        warped = (rng.random((3, H, W)) * 2).astype(np.float32)
        C = 54
        if variant == "full_masked":
            mask = (rng.random((H, W)) < 0.2).astype(np.uint8)
    logits = (rng.standard_normal((C, H, W)) * 1.5).astype(np.float32)
    return noisy, logits, coarse, warped, mask, g


@pytest.mark.parametrize("W,H", [(64, 48), (100, 36), (1920, 1080), (2, 2), (6, 4), (36, 10),
                                 (4, 130)])
@pytest.mark.parametrize("variant", ["coarsest", "mid", "full", "full_masked"])
def test_reconstruct_level_backward_parity(spp, W, H, variant):
    """Frames of every size class: several tiles of 32 x 8 with ragged
    edges, tiny frames whose clamp-to-edge folds many taps onto one
    border pixel (width or height 2), a tile exactly one consumer halo
    wider than the frame."""
    noisy, logits, coarse, warped, mask, g = _level_inputs(W, H, variant, W + H)
    C = logits.shape[0]
    gl = torch.empty((C, H, W), device="cuda")
    gn = torch.zeros((3, H, W), device="cuda")
    gc = None if coarse is None else torch.zeros((3, H // 2, W // 2), device="cuda")
    gw = None if warped is None else torch.zeros((3, H, W), device="cuda")
    spp.check(spp.binding.spp_reconstruct_level_backward(
        dev(noisy), dev(logits), C, None if coarse is None else dev(coarse),
        None if warped is None else dev(warped), None if mask is None else dev(mask), W, H,
        dev(g), gl, gn, gc, gw))
    torch.cuda.synchronize()
    rl, rn, rc, rw = oracle.reconstruct_level_backward(noisy, logits, g, coarse=coarse,
                                                        warped=warped, mask=mask)
    assert_grad(host(gl), rl, "grad logits")
    assert_grad(host(gn), rn, "grad noisy")
    if coarse is not None:
        assert_grad(host(gc), rc, "grad coarse")
    if warped is not None:
        assert_grad(host(gw), rw, "grad warped")


def test_reconstruct_level_backward_coarsest_1x1(spp):
    """A 1 x 1 level: every tap clamps to the one pixel."""
    test_reconstruct_level_backward_parity(spp, 1, 1, "coarsest")
    test_reconstruct_level_backward_parity(spp, 3, 1, "coarsest")


def test_reconstruct_level_backward_is_deterministic(spp):
    """Each gradient element has one writer summing in a fixed order: two
    calls give the same bits."""
    W, H = 640, 360
    noisy, logits, coarse, warped, mask, g = _level_inputs(W, H, "full_masked", 7)
    outs = []
    for _ in range(2):
        gl = torch.empty((54, H, W), device="cuda")
        gn = torch.zeros((3, H, W), device="cuda")
        gc = torch.zeros((3, H // 2, W // 2), device="cuda")
        gw = torch.zeros((3, H, W), device="cuda")
        spp.check(spp.binding.spp_reconstruct_level_backward(
            dev(noisy), dev(logits), 54, dev(coarse), dev(warped), dev(mask), W, H, dev(g), gl,
            gn, gc, gw))
        outs.append((gl, gn, gc, gw))
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_warp_backward_parity(spp):
    W, H = 257, 131
    rng = np.random.default_rng(7)
    mv = ((rng.random((2, H, W)) - 0.5) * 20).astype(np.float32)
    g = rng.standard_normal((3, H, W)).astype(np.float32)
    gp = torch.zeros((3, H, W), device="cuda")
    spp.check(spp.binding.spp_warp_previous_backward(dev(mv), W, H, dev(g), gp))
    assert_grad(host(gp), oracle.warp_backward(mv, g), "grad prev")


def test_tonemap_backward_parity(spp):
    W, H = 300, 200
    rng = np.random.default_rng(8)
    hdr = np.exp(rng.standard_normal((3, H, W)) * 1.5).astype(np.float32)
    gl = rng.standard_normal((3, H, W)).astype(np.float32)
    tm = spp.make_tonemap(1.1, 0.8, 0.2, 0.4, 0.6)
    gh = torch.zeros((3, H, W), device="cuda")
    spp.check(spp.binding.spp_tonemap_backward(dev(hdr), W, H, tm, dev(gl), gh))
    ref = oracle.tonemap_backward(hdr, gl, 1.1, 0.8, 0.2, 0.4, 0.6)
    assert_grad(host(gh), ref, "grad hdr")


def test_l1_loss_parity(spp):
    rng = np.random.default_rng(9)
    a = rng.random(100_003).astype(np.float32)
    b = rng.random(100_003).astype(np.float32)
    loss = torch.zeros(4, device="cuda")[:1]
    grad = torch.empty(100_003, device="cuda")
    spp.check(spp.binding.spp_l1_loss(dev(a), dev(b), a.size, loss, grad))
    v, g = oracle.l1_loss(a, b)
    assert abs(float(loss.item()) - v) <= 1e-5 * v
    assert np.array_equal(np.sign(host(grad)), np.sign(g))
    assert_grad(host(grad), g, "grad l1")


def test_pyramid_backward_parity(spp):
    W, H, L = 96, 64, 4
    rng = np.random.default_rng(10)
    gls = [rng.standard_normal((3, H >> l, W >> l)).astype(np.float32) for l in range(L)]
    g0 = dev(gls[0].copy())
    spp.check(spp.binding.spp_pyramid_backward([dev(x) for x in gls], W, H, L, g0))
    assert_grad(host(g0), oracle.pyramid_backward(gls, W, H), "grad L0")


@pytest.mark.parametrize("hard", [False, True])
def test_splat_backward_parity(spp, hard):
    """Inputs built by the oracle (counts, offsets, samples) and rounded to
    FP32; both sides get the same s, so p = s - floor(s) agrees exactly."""
    W, H = 128, 96
    N = W * H
    rng = np.random.default_rng(11)
    d = np.exp(rng.standard_normal(N)).astype(np.float32)
    seed, frame, lam = 0x5EED, 4, 10.0
    a = oracle.alloc(d, 0.5, lam=lam, hard=hard, seed=seed, frame=frame)
    s32 = a.s.astype(np.float32)
    a.s = s32.astype(np.float64)
    rgb = (rng.random((a.T, 3)) + 0.1).astype(np.float32)
    u = np.array([oracle.pixel_uniform(seed, frame, i) for i in range(N)])
    w = np.array([oracle.assign_one(float(a.s[i]), float(u[i]), lam, hard)[1] for i in range(N)])
    L0 = oracle.splat(a.offsets, rgb, a.s, w, a.extra, W, H, 1)[0]
    g = rng.standard_normal((3, H, W)).astype(np.float32)
    ref = oracle.splat_backward(a, rgb, L0, g, lam=lam, hard=hard, seed=seed, frame=frame)
    rgb4 = np.zeros((a.T, 4), np.float32)
    rgb4[:, :3] = rgb
    gs = torch.empty(N, device="cuda")
    params = spp.make_params(0.5, lam=lam, seed=seed, frame=frame, hard=hard)
    spp.check(spp.binding.spp_splat_backward(
        dev(a.offsets.astype(np.int32)), dev(a.counts.astype(np.int32)), dev(rgb4), dev(s32),
        dev(L0.astype(np.float32)), dev(g), a.T, W, H, params, gs))
    got = host(gs)
    # pixels whose ramp position sits within FP32 rounding of a corner may
    # legitimately take the other side; skip those
    p = a.s - np.floor(a.s)
    r = np.where(p > 0, lam / np.maximum(p, 1e-30) * (u + p - 1), -1)
    near = (np.abs(r) < 1e-3) | (np.abs(r - 1) < 1e-3)
    assert_grad(got[~near], ref[~near], "grad s")


def test_density_backward_parity(spp):
    N = 1 << 16
    rng = np.random.default_rng(12)
    z = rng.standard_normal(N)
    d = np.exp(z - z.max()).astype(np.float32)
    g = rng.standard_normal(N).astype(np.float32)
    gz = torch.empty(N, device="cuda")
    ws = torch.empty(spp.binding.spp_density_backward_workspace_bytes(), dtype=torch.uint8,
                     device="cuda")
    spp.check(spp.binding.spp_density_backward(dev(d), N, 0.25, 0.125, dev(g), gz, ws))
    assert_grad(host(gz), oracle.density_backward(z, g, 0.25), "grad z")
    # the sums are taken in a fixed order: a second call gives the same bits
    gz2 = torch.empty(N, device="cuda")
    spp.check(spp.binding.spp_density_backward(dev(d), N, 0.25, 0.125, dev(g), gz2, ws))
    assert torch.equal(gz, gz2)
    # a workspace below the stated size is refused
    small = torch.empty(256, dtype=torch.uint8, device="cuda")
    assert spp.binding.spp_density_backward(dev(d), N, 0.25, 0.125, dev(g), gz, small) == \
        spp.binding.SPP_ERR_WORKSPACE


def test_autograd_chain_matches_oracle_chain(spp):
    """loss = L1(sRGB(recon(splat(s(z)), logits)), ref) on a 64 x 64 frame
    with 3 levels and the temporal term: gradients with respect to the
    sampler logits z and the kernel logits through the autograd wrappers,
    against the oracle's backward functions composed by hand."""
    from paper_2602_08642_gb300 import autograd as AG
    W = H = 64
    L, B_ = 3, 0.5
    N = W * H
    x = inp.frame_inputs(W, H, L, frame=2, temporal=True)
    rng = np.random.default_rng(13)
    z = rng.standard_normal(N).astype(np.float32)
    d = np.exp(z - z.max()).astype(np.float32)
    prev = (rng.random((3, H, W)) * 2).astype(np.float32)
    ref_img = (rng.random((3, H, W))).astype(np.float32)
    params = spp.make_params(B_, frame=2)
    fr = spp.Frame(W, H, L, max_budget=B_)
    fr.alloc(dev(d), params)
    fr.render(dev(x["clean"]), 0xC0FFEE, 2)
    fr.splat()
    zt = dev(z).requires_grad_(True)
    lgt = [dev(a).requires_grad_(True) for a in x["logits"]]
    s = AG.DensityToS.apply(dev(d), fr.s, B_, 0.125, zt)
    layers = AG.Splat.apply(fr, params, s)
    warped = AG.WarpPrevious.apply(dev(prev), dev(x["mv"]))
    tm = spp.make_tonemap()
    hdr, ldr = AG.Reconstruct.apply(L, tm, warped, dev(x["mask"]), *layers, *lgt)
    loss = AG.L1Loss.apply(ldr, dev(ref_img))
    loss.backward()
    torch.cuda.synchronize()

    # the oracle, composed by hand on its own forward values
    a = oracle.alloc(d, B_, frame=2)
    rgb = oracle.render(x["clean"], a.offsets, 0xC0FFEE, 2)
    lay = oracle.splat(a.offsets, rgb, a.s, a.w, a.extra, W, H, L)
    lg64 = [q.astype(np.float64) for q in x["logits"]]
    wp = oracle.warp(prev.astype(np.float64), x["mv"])
    hats = [None] * L
    for l in range(L - 1, -1, -1):
        hats[l] = oracle.reconstruct_level(lay[l], lg64[l], coarse=hats[l + 1] if l + 1 < L else None,
                                           warped=wp if l == 0 else None,
                                           mask=x["mask"] if l == 0 else None)
    ldr_ref = oracle.tonemap(hats[0])
    v, g_ldr = oracle.l1_loss(ldr_ref, ref_img)
    assert abs(float(loss.item()) - v) <= 1e-4 * v
    g = oracle.tonemap_backward(hats[0], g_ldr)
    g_layers = [None] * L
    g_logits = [None] * L
    for l in range(L):
        gl_, gn_, gc_, _ = oracle.reconstruct_level_backward(
            lay[l], lg64[l], g, coarse=hats[l + 1] if l + 1 < L else None,
            warped=wp if l == 0 else None, mask=x["mask"] if l == 0 else None)
        g_layers[l], g_logits[l] = gn_, gl_
        g = gc_
    g0 = oracle.pyramid_backward(g_layers, W, H)
    gs = oracle.splat_backward(a, rgb, lay[0], g0, seed=0x5EED, frame=2)
    gz = oracle.density_backward(z.astype(np.float64), gs, B_)
    for l in range(L):
        assert_grad(host(lgt[l].grad), g_logits[l], f"grad logits {l}", rtol=3e-4, afrac=3e-5)
    assert_grad(host(zt.grad), gz, "grad z", rtol=1e-3, afrac=1e-4)


@pytest.mark.parametrize("ws", [1.0, 0.0])
def test_combined_loss_parity(spp, ws):
    """Eq. loss_combined (and, with ws = 0, the temporal error alone) and its
    gradient against the FP64 oracle."""
    import oracle.loss as OL
    rng = np.random.default_rng(14 + int(ws))
    n = 3 * 77 * 53
    I, R, P, Q = (rng.random(n).astype(np.float32) for _ in range(4))
    loss = torch.zeros(4, device="cuda")[:1]
    grad = torch.empty(n, device="cuda")
    spp.check(spp.binding.spp_combined_loss(dev(I), dev(R), dev(P), dev(Q), n, 1.25, ws, loss,
                                            grad))
    v, g = OL.combined_loss(I, R, P, Q, 1.25, ws)
    assert abs(float(loss.item()) - v) <= 1e-5 * v
    got = host(grad)
    # the branch taken may differ where the two terms are within FP32 rounding
    s = ws * np.abs(I.astype(np.float64) - R)
    t = 1.25 * np.abs((I.astype(np.float64) - P) - (R.astype(np.float64) - Q))
    clear = np.abs(t - s) > 1e-6
    assert np.allclose(got[clear], g[clear], rtol=1e-6, atol=0)
