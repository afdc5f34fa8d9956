"""Parity of the gradient-estimator ablations (straight-through and
Gumbel-softmax, Sec. 7) with their oracle (oracle/variants.py), and a
training check of the joint predictor under each estimator.

Tolerances: the Gumbel count map and offsets bit-exact; its weights within
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


@pytest.mark.parametrize("estimator", ["straight_through", "gumbel"])
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
