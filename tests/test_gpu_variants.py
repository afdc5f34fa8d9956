"""Parity of the pipeline variants (Sec. 7 ablations) with their oracles
(oracle/variants.py): the low-resolution density map and the systematic
(exact-integer-total) sample map, both bit-exact (integer results, and FP32
results computed in the same order / the same FP64 operations)."""
import numpy as np
import pytest
import torch

import oracle
import oracle.variants as V
import spp_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spp():
    from conftest import build_spp_lib
    build_spp_lib()
    import paper_2602_08642_gb300 as spp
    torch.cuda.set_device(0)
    oracle.build()
    return spp


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("W,H,f", [(64, 32, 2), (1920, 1080, 2), (1920, 1080, 4), (1920, 1080, 8),
                                   (36, 20, 4)])
def test_density_lowres_bit_exact(spp, W, H, f):
    d = inp.density_lognormal(W, H, seed=W + f).ravel()
    out = torch.empty(W * H, device="cuda")
    spp.binding.check(spp.binding.spp_density_lowres(dev(d), W, H, f, out))
    ref = V.density_lowres(d, W, H, f)
    assert np.array_equal(out.cpu().numpy(), ref)
    # in place, and idempotent
    t = dev(d)
    spp.binding.check(spp.binding.spp_density_lowres(t, W, H, f, t))
    assert np.array_equal(t.cpu().numpy(), ref)
    spp.binding.check(spp.binding.spp_density_lowres(t, W, H, f, t))
    assert np.array_equal(t.cpu().numpy(), ref)


def test_density_lowres_rejects_bad_shapes(spp):
    t = torch.zeros(30 * 20, device="cuda")
    with pytest.raises(spp.binding.SppError):
        spp.binding.check(spp.binding.spp_density_lowres(t, 30, 20, 4, t))
    with pytest.raises(spp.binding.SppError):
        spp.binding.check(spp.binding.spp_density_lowres(t, 30, 20, 3, t))


def test_lowres_density_count_map_bit_exact(spp):
    """Sampling from P d: the GPU's count map equals the oracle's stochastic
    allocation of the oracle's P d."""
    W, H, B = 1920, 1080, 0.25
    d = inp.density_lognormal(W, H, seed=4).astype(np.float32).ravel()
    pd = torch.empty(W * H, device="cuda")
    spp.binding.check(spp.binding.spp_density_lowres(dev(d), W, H, 2, pd))
    fr = spp.Frame(W, H, 3, max_budget=B, device=torch.device("cuda"))
    fr.alloc(pd, spp.make_params(B, seed=0x5EED, frame=3))
    torch.cuda.synchronize()
    fr.check_status()
    ref = oracle.alloc(V.density_lowres(d, W, H, 2), B, seed=0x5EED, frame=3)
    assert np.array_equal(fr.counts.cpu().numpy(), ref.counts)


@pytest.mark.parametrize("W,H,B,hard", [(128, 128, 0.25, False), (100, 37, 1.7, False),
                                        (1920, 1080, 0.25, False), (1920, 1080, 0.125, True),
                                        (3840, 2160, 0.5, False), (7, 3, 0.6, False)])
def test_systematic_sample_map_bit_exact(spp, W, H, B, hard):
    d = inp.density_lognormal(W, H, seed=W + H, sigma=1.5).astype(np.float32).ravel()
    fr = spp.Frame(W, H, 1, max_budget=B + 0.1, device=torch.device("cuda"))
    params = spp.make_params(B, seed=77, frame=5, hard=hard)
    fr.alloc_systematic(dev(d), params)
    torch.cuda.synchronize()
    fr.check_status()
    ref = V.alloc_systematic(d, B, hard=hard, seed=77, frame=5)
    T = int(fr.total.item())
    assert T == ref.T
    assert abs(T - B * W * H) < 1 + W * H * 2.0 ** -32
    assert np.array_equal(fr.counts.cpu().numpy(), ref.counts)
    assert np.array_equal(fr.offsets.cpu().numpy(), ref.offsets)
    sp = fr.sample_pixel.cpu().numpy()[:T]
    assert np.array_equal(sp, np.repeat(np.arange(W * H), ref.counts))
    assert np.array_equal(fr.s.cpu().numpy(), ref.s.astype(np.float32))
    w = fr.holdout_w.cpu().numpy()
    assert np.array_equal(w[ref.extra], ref.w[ref.extra])


def test_systematic_total_is_fixed_while_the_stochastic_one_varies(spp):
    """Over ten frames the systematic total stays within one sample of B N
    while the stochastic total spreads by about sqrt(B N (1 - B))."""
    W, H, B = 256, 256, 0.25
    d = inp.density_lognormal(W, H, seed=8).astype(np.float32).ravel()
    fr = spp.Frame(W, H, 1, max_budget=0.5, device=torch.device("cuda"))
    t_sys, t_sto = [], []
    for k in range(10):
        fr.alloc_systematic(dev(d), spp.make_params(B, seed=5, frame=k))
        t_sys.append(int(fr.total.item()))
        fr.alloc(dev(d), spp.make_params(B, seed=5, frame=k))
        t_sto.append(int(fr.total.item()))
    assert max(abs(t - B * W * H) for t in t_sys) < 1.001
    assert np.std(t_sto) > 20


def test_two_stage_with_the_variants(spp):
    """The two-stage pipeline trains with the low-resolution density map (the
    density it samples from is block-constant, the gradient goes back through
    P) and runs inference with the systematic sample map (its total within
    one sample of B N on every frame)."""
    import oracle.unet as U
    from paper_2602_08642_gb300 import learned as Lm
    from paper_2602_08642_gb300 import two_stage as T2
    size, budget = 64, 0.25
    train = [Lm.FrameData(inp.training_pair(size, seed=100 + i)) for i in range(8)]
    fb = inp.fixed_head_bias()
    ts = torch.from_numpy(inp.unet_params(U.layers("sampler"), seed=3))
    td = torch.from_numpy(inp.unet_params(
        U.layers("denoiser"), seed=4,
        head_bias={"h0": np.concatenate([fb["h0"][:54], np.zeros(10, np.float32)]),
                   "h1": fb["h1"], "h2": fb["h2"]}))
    tr = T2.TwoStageTrainer(ts, td, 4, size, budget, lr=1e-3, density_factor=2)
    losses = [tr.step(train[4 * (k % 2):4 * (k % 2) + 4], seed=k) for k in range(20)]
    assert np.all(np.isfinite(losses))
    dl = tr.p.d_lr[0].cpu().numpy()
    assert np.array_equal(dl, np.repeat(np.repeat(dl[::2, ::2], 2, 0), 2, 1))
    assert np.any(tr.p.sampler.grad.cpu().numpy() != 0)
    p = T2.TwoStage(tr.p.sampler.theta, tr.p.denoiser.theta, 1, size, size, budget,
                    rounding="systematic")
    s = train[0]
    p.begin_sequence()
    for k, (g, c) in enumerate([(s.gprev, s.clean_prev), (s.g, s.clean)]):
        p.frame([g], [s.mv], [c], 9, k)
        assert abs(int(p.frames[0].total.item()) - budget * size * size) < 1.001
