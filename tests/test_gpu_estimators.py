"""Parity of the gradient-estimator ablations (straight-through,
Gumbel-softmax and the DASR surrogate of Sec. 4.1; Sec. 7) with their oracle
(oracle/variants.py), and a training check of the joint predictor under
each estimator.

Tolerances: the Gumbel and DASR count maps and offsets bit-exact; the DASR
splat 1e-5 relative (an FP32 sum of at most a few samples, one division);
the Gumbel weights within
1e-6 relative (FP64 log / exp of two libraries, then FP32 rounding); the
gradients as the relaxed splat backward's (1e-4 relative + 1e-5 of the
largest magnitude), the straight-through's rendered samples being FP32."""
import numpy as np
import pytest
import torch

import oracle
import oracle.variants as V
import spp_inputs as inp
from test_gpu_backward import assert_grad

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spp():
    from conftest import build_spp_lib
    build_spp_lib()
    import paper_2602_08642_gb300 as spp
    torch.cuda.set_device(0)
    oracle.build()
    return spp


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("W,H,B", [(128, 96, 0.5), (100, 37, 1.3), (1920, 1080, 0.25)])
def test_gumbel_sample_map_parity(spp, W, H, B):
    d = inp.density_lognormal(W, H, seed=W).ravel()
    lam, seed, frame = 10.0, 0x5EED, 6
    fr = spp.Frame(W, H, 1, max_budget=B + 1.0, device=torch.device("cuda"))
    fr.alloc(dev(d), spp.make_params(B, lam=lam, seed=seed, frame=frame, gumbel=True))
    torch.cuda.synchronize()
    fr.check_status()
    ref = V.alloc_gumbel(d, B, lam=lam, seed=seed, frame=frame)
    assert int(fr.total.item()) == ref.T
    assert np.array_equal(fr.counts.cpu().numpy(), ref.counts)
    assert np.array_equal(fr.offsets.cpu().numpy(), ref.offsets)
    assert np.array_equal(fr.s.cpu().numpy(), ref.s.astype(np.float32))
    w = host(fr.holdout_w)
    e = ref.extra
    assert np.allclose(w[e], ref.w[e].astype(np.float64), rtol=1e-6, atol=1e-30)


@pytest.mark.parametrize("estimator", ["gumbel", "straight_through"])
def test_estimator_backward_parity(spp, estimator):
    """Inputs built by the oracle (sample map, samples, L^0) and rounded to
    FP32; both sides get the same s."""
    W, H = 128, 96
    N = W * H
    rng = np.random.default_rng(13)
    d = np.exp(rng.standard_normal(N)).astype(np.float32)
    seed, frame, lam, rseed = 0x5EED, 4, 10.0, 0xC0FFEE
    clean, _ = inp.scene(W, H, seed=3)
    if estimator == "gumbel":
        a = V.alloc_gumbel(d, 0.5, lam=lam, seed=seed, frame=frame)
        params = spp.make_params(0.5, lam=lam, seed=seed, frame=frame, gumbel=True)
        est = spp.binding.SPP_ESTIMATOR_GUMBEL
    else:
        a = oracle.alloc(d, 0.5, hard=True, seed=seed, frame=frame)
        params = spp.make_params(0.5, seed=seed, frame=frame, hard=True)
        est = spp.binding.SPP_ESTIMATOR_STRAIGHT_THROUGH
    s32 = a.s.astype(np.float32)
    a.s = s32.astype(np.float64)
    a.p = a.s - np.floor(a.s)
    rgb = oracle.render(clean, a.offsets, rseed, frame).astype(np.float32)
    L0 = oracle.splat(a.offsets, rgb, a.s, a.w, a.extra, W, H, 1)[0]
    g = rng.standard_normal((3, H, W)).astype(np.float32)
    ref = V.splat_backward_estimator(a, rgb, L0, g, estimator, lam=lam,
                                     clean=clean.astype(np.float32), render_seed=rseed,
                                     frame=frame)
    rgb4 = np.zeros((a.T, 4), np.float32)
    rgb4[:, :3] = rgb
    gs = torch.empty(N, device="cuda")
    spp.check(spp.binding.spp_splat_backward_estimator(
        dev(a.offsets.astype(np.int32)), dev(a.counts.astype(np.int32)), dev(rgb4), dev(s32),
        dev(L0.astype(np.float32)), dev(g), dev(np.asarray(a.w, np.float32)), a.T, W, H, params,
        est, dev(clean.astype(np.float32)), rseed, gs))
    assert_grad(host(gs), ref, f"grad s ({estimator})", rtol=1e-4, afrac=1e-5)


@pytest.mark.parametrize("W,H,B", [(128, 96, 0.5), (100, 37, 1.3), (1920, 1080, 0.25)])
def test_dasr_sample_map_parity(spp, W, H, B):
    """The deterministic rounding of Sec. 4.1 (Eq. kuz_fw): count map,
    offsets and total bit-exact with the oracle; s_out carries the splat's
    normaliser max(n, 1) and every holdout weight is 1."""
    d = inp.density_lognormal(W, H, seed=W + 3).ravel()
    fr = spp.Frame(W, H, 1, max_budget=B + 0.5, device=torch.device("cuda"))
    fr.alloc(dev(d), spp.make_params(B, frame=3, dasr=True))
    torch.cuda.synchronize()
    fr.check_status()
    ref = V.alloc_dasr(d, B)
    assert int(fr.total.item()) == ref.T
    assert np.array_equal(fr.counts.cpu().numpy(), ref.counts)
    assert np.array_equal(fr.offsets.cpu().numpy(), ref.offsets)
    assert np.array_equal(fr.s.cpu().numpy(), ref.norm.astype(np.float32))
    assert torch.all(fr.holdout_w == 1.0)


def test_dasr_sample_map_rounds_exact_halves_up(spp):
    """A uniform density puts s = B = 2.5 exactly on every pixel: each gets
    three samples."""
    W, H = 64, 64
    fr = spp.Frame(W, H, 1, max_budget=3.0, device=torch.device("cuda"))
    fr.alloc(torch.ones(H, W, device="cuda"), spp.make_params(2.5, dasr=True))
    torch.cuda.synchronize()
    fr.check_status()
    assert torch.all(fr.counts == 3) and int(fr.total.item()) == 3 * W * H


def test_dasr_splat_parity(spp):
    """Eq. kuz_fw through the library's renderer stand-in and splat: the
    per-pixel sample mean (0 without samples) and its pyramid, against the
    oracle on the same samples."""
    W, H, L, B = 160, 96, 3, 0.3
    d = inp.density_lognormal(W, H, seed=17).ravel()
    clean, _ = inp.scene(W, H, seed=5)
    fr = spp.Frame(W, H, L, max_budget=B + 0.5, device=torch.device("cuda"))
    fr.alloc(dev(d), spp.make_params(B, frame=2, dasr=True))
    fr.render(dev(clean), 0xC0FFEE, 2)
    fr.splat()
    torch.cuda.synchronize()
    fr.check_status()
    T = int(fr.total.item())
    rgb = host(fr.rgb[:T, :3])
    ref = V.splat_dasr(fr.counts.cpu().numpy(), rgb, W, H, L)
    assert np.any(fr.counts.cpu().numpy() == 0) and np.any(fr.counts.cpu().numpy() >= 2)
    for l in range(L):
        got = host(fr.layers[l])
        assert np.all(np.abs(got - ref[l]) <= 1e-5 * np.abs(ref[l])), l
        if l == 0:
            assert np.all(got[:, fr.counts.cpu().numpy().reshape(H, W) == 0] == 0)


def test_dasr_backward_parity(spp):
    """The surrogate gradient of Eq. kuz_grad against the oracle (the
    tolerance of the other splat gradients)."""
    W, H, B = 128, 96, 0.4
    N = W * H
    rng = np.random.default_rng(19)
    d = np.exp(rng.standard_normal(N)).astype(np.float32)
    clean, _ = inp.scene(W, H, seed=6)
    a = V.alloc_dasr(d, B)
    rgb = oracle.render(clean, a.offsets, 0xC0FFEE, 1).astype(np.float32)
    L0 = V.splat_dasr(a.counts, rgb, W, H, 1)[0].astype(np.float32)
    g = rng.standard_normal((3, H, W)).astype(np.float32)
    ref_img = clean.astype(np.float32)
    want = V.splat_backward_dasr(a.counts, L0, g, ref_img)
    gs = torch.empty(N, device="cuda")
    params = spp.make_params(B, dasr=True)
    rgb4 = np.zeros((a.T, 4), np.float32)
    rgb4[:, :3] = rgb
    spp.check(spp.binding.spp_splat_backward_estimator(
        dev(a.offsets.astype(np.int32)), dev(a.counts.astype(np.int32)), dev(rgb4),
        dev(a.norm.astype(np.float32)), dev(L0), dev(g), None, a.T, W, H, params,
        spp.binding.SPP_ESTIMATOR_DASR, dev(ref_img), 0, gs))
    assert_grad(host(gs), want, "grad s (DASR)", rtol=1e-4, afrac=1e-5)
    # the unsampled pixels get the reference alone
    z = a.counts == 0
    assert np.allclose(host(gs)[z], (g.reshape(3, -1) * ref_img.reshape(3, -1)).sum(0)[z],
                       rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("estimator", ["straight_through", "gumbel", "dasr"])
def test_training_under_each_estimator(spp, estimator):
    """The joint predictor trains under each estimator (the Gumbel forward
    traces every extra sample, the straight-through forward is hard); the
    trained model runs the hard test-time rule."""
    import oracle.unet as U
    from paper_2602_08642_gb300 import learned as Lm
    size, budget = 64, 0.25
    train = [Lm.FrameData(inp.training_pair(size, seed=100 + i)) for i in range(16)]
    theta = torch.from_numpy(inp.unet_params(U.LAYERS, seed=5, head_bias=inp.fixed_head_bias()))
    tr = Lm.Trainer(theta, 8, size, budget, lr=1e-3, estimator=estimator)
    rng = np.random.default_rng(0)
    losses = []
    for k in range(80):
        idx = rng.choice(len(train), 8, replace=False)
        losses.append(tr.step([train[i] for i in idx], seed=1000 + 17 * k))
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-20:]) < np.mean(losses[:20])
    held = [Lm.FrameData(inp.training_pair(size, seed=900 + i)) for i in range(4)]
    psnr = Lm.evaluate(held, budget, tr.net.theta, None, estimator=estimator)
    assert np.all(np.isfinite(psnr))
