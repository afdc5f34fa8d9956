"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances, written here and derived in the design notes:
  - integer work (counts, offsets, sample list, T): bit-exact;
  - FP32 outputs: relative error <= 1e-5 per element (every output is a sum
    of non-negative terms, so relative error is meaningful; exact zeros must
    stay exact zeros);
  - tone-mapped sRGB: relative 1e-5 plus absolute 1e-6.
Inputs come from the seeded generator in ``spp_inputs``; the oracle never
sees a value the CUDA path produced.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import spp_inputs as inp

pytestmark = pytest.mark.gpu

RTOL = 1e-5
LDR_ATOL = 1e-6


@pytest.fixture(scope="module")
def spp():
    from conftest import build_spp_lib
    build_spp_lib()
    import paper_2602_08642_gb300 as spp
    torch.cuda.set_device(0)
    return spp


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def assert_rel(got, ref, rtol=RTOL, atol=0.0, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    err = np.abs(got - ref)
    bound = rtol * np.abs(ref) + atol
    bad = err > bound
    if bad.any():
        k = np.argmax(err / np.maximum(bound, 1e-300))
        raise AssertionError(f"{what}: {bad.sum()} elements out of tolerance; worst at flat "
                             f"index {k}: got {got.ravel()[k]!r} ref {ref.ravel()[k]!r}")
    # exact zeros stay exact zeros
    assert np.all(got[ref == 0.0] == 0.0), what


def run_alloc(spp, d, W, H, params, capacity=None):
    fr = spp.Frame(W, H, 1, max_budget=max(params.budget, 0.01), capacity=capacity)
    fr.clear_status()
    fr.alloc(dev(d), params)
    torch.cuda.synchronize()
    return fr


def oracle_alloc(d, params):
    return oracle.alloc(d, params.budget, phi=params.uniform_fraction, lam=params.lambda_,
                        hard=params.holdout_mode == 1, seed=params.seed, frame=params.frame)


def check_alloc(fr, ref, what=""):
    N = fr.N
    T = fr.sample_count()
    assert T == ref.T, what
    assert np.array_equal(host(fr.counts), ref.counts), what
    assert np.array_equal(host(fr.offsets), ref.offsets), what
    assert np.array_equal(host(fr.sample_pixel)[:T], ref.sample_pixel), what
    s = host(fr.s).astype(np.float64)
    assert np.all(np.abs(s - ref.s) <= 2.0**-23 * ref.s), what
    assert_rel(host(fr.holdout_w), ref.w, what=what + " holdout_w")
    assert N == ref.counts.size


# ---------------------------------------------------------------------------
# a1-a3: count map, offsets, sample list
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("W,H", [(1, 1), (7, 5), (128, 128), (97, 61), (1000, 700),
                                 (1920, 1080)])
@pytest.mark.parametrize("B,hard", [(0.25, False), (0.11, True), (4.0, False)])
def test_alloc_bit_exact(spp, W, H, B, hard):
    d = inp.density_lognormal(W, H, seed=W * 7 + H)
    params = spp.make_params(B, seed=0x5EED + W, frame=3, hard=hard)
    fr = run_alloc(spp, d, W, H, params)
    assert fr.check_status() == 0
    check_alloc(fr, oracle_alloc(d, params), f"{W}x{H} B={B}")


def test_alloc_bit_exact_4k(spp):
    """The 4K frame: many pixels per CTA of the one-launch sample map."""
    W, H = 3840, 2160
    d = inp.density_lognormal(W, H, seed=44)
    params = spp.make_params(0.125, seed=0x5EED, frame=9)
    fr = run_alloc(spp, d, W, H, params)
    assert fr.check_status() == 0
    check_alloc(fr, oracle_alloc(d, params), "4K")


def test_alloc_workspace_in_any_prior_state(spp):
    """The sample map clears what it needs: a workspace filled with random
    bytes, then reused call after call (with different frame sizes), gives
    the oracle's map every time."""
    fr = spp.Frame(1920, 1080, 1, max_budget=0.5)
    g = torch.Generator(device="cuda").manual_seed(5)
    fr.alloc_ws.copy_(torch.randint(0, 256, fr.alloc_ws.shape, generator=g, device="cuda",
                                    dtype=torch.int32).to(torch.uint8))
    for k, (W, H) in enumerate([(1920, 1080), (300, 200), (1920, 1080), (64, 64)]):
        d = inp.density_lognormal(W, H, seed=90 + k)
        params = spp.make_params(0.5, frame=k)
        small = spp.Frame(W, H, 1, max_budget=0.5)
        small.alloc_ws = fr.alloc_ws  # one workspace for every call
        small.clear_status()
        small.alloc(dev(d), params)
        torch.cuda.synchronize()
        assert small.check_status() == 0
        check_alloc(small, oracle_alloc(d, params), f"reused workspace, call {k}")


def test_alloc_without_count_map(spp):
    """counts = NULL: the offsets and the sample list come from the same
    decisions taken again."""
    W, H = 1000, 700
    d = inp.density_lognormal(W, H, seed=12)
    params = spp.make_params(0.6, frame=2)
    ref = run_alloc(spp, d, W, H, params)
    fr = spp.Frame(W, H, 1, max_budget=0.6)
    fr.clear_status()
    spp.check(spp.spp_alloc_sample_map(dev(d), W, H, params, None, fr.offsets, fr.sample_pixel,
                                       fr.capacity, fr.s, fr.holdout_w, fr.total, fr.status,
                                       fr.alloc_ws))
    torch.cuda.synchronize()
    assert fr.check_status() == 0
    T = ref.sample_count()
    assert fr.sample_count() == T
    assert torch.equal(fr.offsets, ref.offsets)
    assert torch.equal(fr.sample_pixel[:T], ref.sample_pixel[:T])
    assert torch.equal(fr.s, ref.s) and torch.equal(fr.holdout_w, ref.holdout_w)


def test_alloc_interleaved_with_systematic_map(spp):
    """The stochastic and the systematic map share one workspace, call
    after call, and each stays exact."""
    import oracle.variants as V
    W, H = 960, 540
    fr = spp.Frame(W, H, 1, max_budget=0.5)
    for k in range(3):
        d = inp.density_lognormal(W, H, seed=60 + k)
        params = spp.make_params(0.25, frame=k)
        fr.clear_status()
        fr.alloc(dev(d), params)
        torch.cuda.synchronize()
        assert fr.check_status() == 0
        check_alloc(fr, oracle_alloc(d, params), f"stochastic {k}")
        fr.alloc_systematic(dev(d), params)
        torch.cuda.synchronize()
        assert fr.check_status() == 0
        ref = V.alloc_systematic(d.ravel(), 0.25, seed=params.seed, frame=k)
        assert np.array_equal(host(fr.counts), ref.counts)


def test_alloc_fp64_path_agrees_with_filter(spp):
    W, H = 640, 480
    d = inp.density_lognormal(W, H, seed=5)
    p1 = spp.make_params(0.5, frame=1)
    p2 = spp.make_params(0.5, frame=1, exact_fp64=True)
    a = run_alloc(spp, d, W, H, p1)
    b = run_alloc(spp, d, W, H, p2)
    assert np.array_equal(host(a.counts), host(b.counts))
    assert np.array_equal(host(a.offsets), host(b.offsets))
    assert_rel(host(a.holdout_w), host(b.holdout_w), rtol=2e-6, what="w filter vs fp64")
    check_alloc(b, oracle_alloc(d, p2), "fp64 path")


def test_alloc_integer_densities_take_fp64_path(spp):
    """Constant d with B = 1 gives s_i = 1 exactly (1/8 + 7/8): p = 0, every
    pixel sits on the integer threshold and one sample each is taken."""
    W, H = 300, 200
    d = np.full((H, W), 2.5, np.float32)
    params = spp.make_params(1.0)
    fr = run_alloc(spp, d, W, H, params)
    ref = oracle_alloc(d, params)
    assert np.all(ref.counts == 1)
    check_alloc(fr, ref, "integer s")


def test_alloc_wide_dynamic_range_density(spp):
    """The exact sum covers the whole FP32 range: subnormals, zeros and values
    near FLT_MAX / N in one map."""
    W, H = 513, 259
    rng = np.random.default_rng(3)
    e = rng.integers(-149, 100, size=(H, W))
    d = np.ldexp(1.0 + rng.random((H, W)), e).astype(np.float32)
    d[rng.random((H, W)) < 0.1] = 0.0
    d[rng.random((H, W)) < 0.01] = np.float32(1.4e-45)
    params = spp.make_params(0.25, frame=9)
    fr = run_alloc(spp, d, W, H, params)
    ref = oracle_alloc(d, params)
    assert ref.S == math.fsum(d.astype(np.float64).ravel().tolist())
    check_alloc(fr, ref, "wide range")


@pytest.mark.parametrize("e_lo,width", [(1, 33), (100, 32), (220, 33)])
def test_alloc_exponent_bands(spp, e_lo, width):
    """Densities whose exponents fill a band of `width` binades (plus 5 %
    zeros), at the bottom of the normal range, in the middle and near the
    top: the chunks of 8 values a thread sums in 64 bits at once span up to
    32 binades (the exact-sum fast path) or 33 (the per-value path), both in
    the same threads, several chunks per thread at 4096 x 2048."""
    W, H = 4096, 2048
    rng = np.random.default_rng(11 + e_lo)
    e = rng.integers(e_lo, e_lo + width + 1, size=(H, W))
    d = np.ldexp(1.0 + rng.random((H, W)), e - 127).astype(np.float32)
    d[rng.random((H, W)) < 0.05] = 0.0
    params = spp.make_params(0.25, frame=3)
    fr = run_alloc(spp, d, W, H, params)
    ref = oracle_alloc(d, params)
    assert ref.S == math.fsum(d.astype(np.float64).ravel().tolist())
    check_alloc(fr, ref, f"band {e_lo}+{width}")


def test_alloc_phi_zero_and_one(spp):
    W, H = 256, 64
    d = inp.density_lognormal(W, H, seed=8)
    for phi in (0.0, 1.0):
        params = spp.make_params(0.5, uniform_fraction=phi, frame=2)
        fr = run_alloc(spp, d, W, H, params)
        check_alloc(fr, oracle_alloc(d, params), f"phi={phi}")


@pytest.mark.parametrize("bad", [np.nan, -1.0, np.inf])
def test_alloc_rejects_bad_density(spp, bad):
    W, H = 64, 64
    d = inp.density_lognormal(W, H, seed=1)
    d[10, 20] = bad
    fr = run_alloc(spp, d, W, H, spp.make_params(0.25))
    assert spp.spp_get_status(fr.status) == spp.binding.SPP_ERR_INPUT
    assert fr.sample_count() == 0
    assert np.all(host(fr.offsets) == 0)


def test_alloc_all_zero_density(spp):
    fr = run_alloc(spp, np.zeros((32, 32), np.float32), 32, 32, spp.make_params(0.25))
    assert spp.spp_get_status(fr.status) == spp.binding.SPP_ERR_INPUT


def test_alloc_capacity_overflow_is_reported_not_written(spp):
    W, H = 256, 256
    d = inp.density_lognormal(W, H, seed=2)
    params = spp.make_params(0.5)
    ref = oracle_alloc(d, params)
    cap = ref.T // 2
    fr = spp.Frame(W, H, 1, capacity=ref.T + 1024)
    fr.sample_pixel.fill_(-7)
    fr.clear_status()
    spp.check(spp.spp_alloc_sample_map(dev(d), W, H, params, fr.counts, fr.offsets,
                                       fr.sample_pixel, cap, fr.s, fr.holdout_w, fr.total,
                                       fr.status, fr.alloc_ws))
    torch.cuda.synchronize()
    assert spp.spp_get_status(fr.status) == spp.binding.SPP_ERR_CAPACITY
    sp = host(fr.sample_pixel)
    assert np.array_equal(sp[:cap], ref.sample_pixel[:cap])
    assert np.all(sp[cap:] == -7)
    assert fr.sample_count() == ref.T


def test_alloc_empty_frame(spp):
    fr = spp.Frame(0, 0, 1, capacity=16)
    fr.offsets.fill_(5)
    fr.alloc(torch.zeros(4, device="cuda"), spp.make_params(0.25))
    torch.cuda.synchronize()
    assert fr.sample_count() == 0 and int(fr.offsets[0]) == 0


def test_alloc_bounded_wait_reports_timeout(spp):
    """A scan tile that never publishes makes the later tiles' look-back waits
    run out: the kernel returns, the status says SPP_ERR_TIMEOUT, and the
    context stays usable for the next call."""
    W, H = 64, 256  # 8 scan tiles
    d = inp.density_lognormal(W, H, seed=4)
    params = spp.make_params(0.25)
    params.flags |= spp.binding.SPP_FLAG_TEST_STALL_TILE1
    fr = run_alloc(spp, d, W, H, params)
    assert spp.spp_get_status(fr.status) == spp.binding.SPP_ERR_TIMEOUT
    good = run_alloc(spp, d, W, H, spp.make_params(0.25))
    assert good.check_status() == 0
    check_alloc(good, oracle_alloc(d, spp.make_params(0.25)), "after timeout")


def test_alloc_deterministic(spp):
    W, H = 1920, 1080
    d = inp.density_lognormal(W, H, seed=6)
    params = spp.make_params(0.25, frame=4)
    a = run_alloc(spp, d, W, H, params)
    b = run_alloc(spp, d, W, H, params)
    for x, y in [(a.counts, b.counts), (a.offsets, b.offsets), (a.s, b.s),
                 (a.holdout_w, b.holdout_w)]:
        assert torch.equal(x, y)


def test_alloc_sample_count_statistics(spp):
    """E[T] = B N over frames (Sec. 3)."""
    W, H = 512, 512
    d = inp.density_lognormal(W, H, seed=11)
    fr = spp.Frame(W, H, 1, max_budget=0.25)
    Ts = []
    for t in range(64):
        fr.alloc(dev(d), spp.make_params(0.25, frame=t))
        Ts.append(fr.sample_count())
    s = host(fr.s).astype(np.float64)
    p = s - np.floor(s)
    sigma = math.sqrt(float((p * (1 - p)).sum()))
    assert abs(np.mean(Ts) - 0.25 * W * H) < 4.5 * sigma / math.sqrt(len(Ts))


# ---------------------------------------------------------------------------
# a4-a5: renderer stand-in, splat and pyramid
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("W,H,L,B", [(128, 128, 2, 0.25), (200, 72, 3, 0.5), (1920, 1080, 3, 0.25),
                                     (64, 48, 5, 4.0)])
def test_render_and_splat_parity(spp, W, H, L, B):
    d = inp.density_lognormal(W, H, seed=21)
    clean, _ = inp.scene(W, H, seed=22)
    params = spp.make_params(B, frame=5)
    fr = spp.Frame(W, H, L, max_budget=B)
    fr.clear_status()
    fr.alloc(dev(d), params)
    fr.render(dev(clean), 0xC0FFEE, 5)
    fr.splat()
    torch.cuda.synchronize()
    assert fr.check_status() == 0
    ref = oracle_alloc(d, params)
    check_alloc(fr, ref, "alloc before splat")
    rgb_ref = oracle.render(clean, ref.offsets, 0xC0FFEE, 5)
    rgb = host(fr.rgb)[: ref.T]
    assert_rel(rgb[:, :3], rgb_ref, what="render")
    assert np.all(rgb[:, 3] == 0)
    layers_ref = oracle.splat(ref.offsets, rgb_ref, ref.s, ref.w, ref.extra, W, H, L)
    for l in range(L):
        assert_rel(host(fr.layers[l]), layers_ref[l], what=f"layer {l}")


# ---------------------------------------------------------------------------
# a6-a9: reconstruction levels and tone map
# ---------------------------------------------------------------------------
def _recon_inputs(W, H, L, seed, temporal=True, C0=None):
    rng = np.random.default_rng(seed)
    layers = [(rng.random((3, H >> l, W >> l)) * 3).astype(np.float32) for l in range(L)]
    # some exact zeros, as in a sparse splat
    layers[0][:, rng.random((H, W)) < 0.6] = 0.0
    lg = inp.random_logits(W, H, L, seed=seed + 1, temporal=temporal)
    prev = (rng.random((3, H, W)) * 3).astype(np.float32)
    mv = inp.motion_affine(W, H, seed=seed + 2)
    mask = inp.disocclusion_mask(W, H, seed=seed + 3, frac=0.1)
    return layers, lg, prev, mv, mask


@pytest.mark.parametrize("W,H,L", [(64, 48, 2), (100, 36, 3), (1920, 1080, 3), (96, 96, 5)])
@pytest.mark.parametrize("temporal", [True, False])
def test_reconstruct_frame_parity(spp, W, H, L, temporal):
    layers, lg, prev, mv, mask = _recon_inputs(W, H, L, 31 + W, temporal)
    tm = spp.make_tonemap(1.1, 0.9, 0.2, 0.4, 0.6)
    fr = spp.Frame(W, H, L, capacity=16)
    for l in range(L):
        fr.layers[l].copy_(dev(layers[l]))
    out = fr.reconstruct([dev(a) for a in lg], prev=dev(prev) if temporal else None,
                         mv=dev(mv), mask=dev(mask), tm=tm)
    torch.cuda.synchronize()
    hdr_ref, hats = oracle.reconstruct([a.astype(np.float64) for a in layers],
                                       [a.astype(np.float64) for a in lg],
                                       prev=prev.astype(np.float64) if temporal else None,
                                       mv=mv, mask=mask)
    assert_rel(host(out), hdr_ref, what="hdr")
    ldr_ref = oracle.tonemap(hdr_ref, 1.1, 0.9, 0.2, 0.4, 0.6)
    assert_rel(host(fr.ldr), ldr_ref, atol=LDR_ATOL, what="ldr")


@pytest.mark.parametrize("W,H", [(1920, 1080), (37, 23)])
def test_warp_previous_parity(spp, W, H):
    """W_t L_{t-1}: bilinear reprojection along the motion vectors, including
    positions clamped at every border and exactly zero motion."""
    rng = np.random.default_rng(61)
    prev = (rng.random((3, H, W)) * 3).astype(np.float32)
    mv = ((rng.random((2, H, W)) - 0.5) * 24).astype(np.float32)
    mv[:, : H // 4] = 0.0
    out = torch.empty((3, H, W), device="cuda")
    spp.check(spp.spp_warp_previous(dev(prev), dev(mv), W, H, out))
    ref = oracle.warp(prev.astype(np.float64), mv)
    assert_rel(host(out), ref, what="warp")
    assert np.array_equal(host(out)[:, : H // 4], prev[:, : H // 4])


def test_reconstruct_level_intermediate_parity(spp):
    W, H = 160, 90
    rng = np.random.default_rng(41)
    noisy = (rng.random((3, H, W)) * 2).astype(np.float32)
    coarse = (rng.random((3, H // 2, W // 2)) * 2).astype(np.float32)
    lg = rng.standard_normal((29, H, W)).astype(np.float32) * 3
    out = torch.empty((3, H, W), device="cuda")
    spp.check(spp.spp_reconstruct_level(dev(noisy), dev(lg), 29, dev(coarse), None, None, W, H,
                                        None, out, None))
    ref = oracle.reconstruct_level(noisy, lg, coarse=coarse)
    assert_rel(host(out), ref, what="mid level")


def test_reconstruct_bounded_wait_reports_timeout(spp):
    """A tile whose copies are never issued makes its CTA's pipeline waits
    run out (about 100 ms): the launch returns, the status says
    SPP_ERR_TIMEOUT, the tiles of the other CTAs are still right, and the
    next call is unaffected."""
    W, H = 960, 540  # level 1 of a 1080p frame: 15 x 135 tiles of 64 x 4
    rng = np.random.default_rng(43)
    noisy = (rng.random((3, H, W)) * 2).astype(np.float32)
    coarse = (rng.random((3, H // 2, W // 2)) * 2).astype(np.float32)
    lg = rng.standard_normal((29, H, W)).astype(np.float32) * 3
    ref = oracle.reconstruct_level(noisy, lg, coarse=coarse)
    tiles_x, tiles = W // 64, (W // 64) * ((H + 3) // 4)
    G = min(torch.cuda.get_device_properties(0).multi_processor_count, tiles)
    stalled = G + 7  # the second tile of CTA 7 (issued in the pipeline's prologue)
    st = torch.zeros(4, dtype=torch.int32, device="cuda")[:1]
    out = torch.full((3, H, W), -1.0, device="cuda")
    assert spp.binding.spp_test_stall_reconstruction(stalled) == 0
    spp.check(spp.spp_reconstruct_level(dev(noisy), dev(lg), 29, dev(coarse), None, None, W, H,
                                        None, out, None, st))
    assert spp.spp_get_status(st) == spp.binding.SPP_ERR_TIMEOUT
    got = host(out)
    t = np.arange(tiles)
    mine = (t % G == 7) & (t >= stalled)  # CTA 7 stops at the stalled tile
    tile_of = (np.arange(H)[:, None] // 4) * tiles_x + np.arange(W)[None, :] // 64
    keep = ~mine[tile_of]
    assert_rel(got[:, keep], ref[:, keep], what="tiles of the other CTAs")
    # the hook is one-shot: the next call runs every tile
    spp.spp_clear_status(st)
    spp.check(spp.spp_reconstruct_level(dev(noisy), dev(lg), 29, dev(coarse), None, None, W, H,
                                        None, out, None, st))
    assert spp.spp_get_status(st) == 0
    assert_rel(host(out), ref, what="after the timeout")


def test_reconstruct_invariants_on_gpu(spp):
    """Constant layers and previous frame give the constant back; one-hot
    centre logits give the identity; zero motion makes W_t the identity."""
    W, H, L = 128, 64, 3
    _, lg, _, mv, mask = _recon_inputs(W, H, L, 51)
    fr = spp.Frame(W, H, L, capacity=16)
    for l in range(L):
        fr.layers[l].fill_(1.75)
    out = fr.reconstruct([dev(a) for a in lg], prev=torch.full((3, H, W), 1.75, device="cuda"),
                         mv=dev(mv), mask=dev(mask))
    torch.cuda.synchronize()
    assert np.allclose(host(out), 1.75, rtol=RTOL, atol=0)
    one_hot = []
    for l in range(L):
        a = np.zeros_like(lg[l])
        a[12] = 60.0
        one_hot.append(a)
    rng = np.random.default_rng(52)
    for l in range(L):
        fr.layers[l].copy_(dev(rng.random((3, H >> l, W >> l)).astype(np.float32)))
    out = fr.reconstruct([dev(a) for a in one_hot], prev=dev(rng.random((3, H, W)).astype(np.float32)),
                         mv=dev(np.zeros((2, H, W), np.float32)), mask=None)
    torch.cuda.synchronize()
    assert_rel(host(out), host(fr.layers[0]), rtol=2e-6, what="one-hot identity")


# ---------------------------------------------------------------------------
# Whole frames through the pipeline
# ---------------------------------------------------------------------------
def _frame_parity(spp, W, H, L, B, temporal, frame_index=1, seed=1):
    x = inp.frame_inputs(W, H, L, frame=frame_index, temporal=temporal, base_seed=seed)
    prev = None
    if temporal:
        prev = (np.random.default_rng(seed).random((3, H, W)) * 2).astype(np.float32)
    params = spp.make_params(B, frame=frame_index)
    fr = spp.Frame(W, H, L, max_budget=B)
    fr.clear_status()
    out = fr.run(dev(x["d"]), dev(x["clean"]), [dev(a) for a in x["logits"]], params,
                 prev=dev(prev) if temporal else None, mv=dev(x["mv"]), mask=dev(x["mask"]))
    torch.cuda.synchronize()
    assert fr.check_status() == 0
    ref = oracle.frame(x["d"], x["clean"], [a.astype(np.float64) for a in x["logits"]], W, H, L,
                       B, prev=None if prev is None else prev.astype(np.float64), mv=x["mv"],
                       mask=x["mask"], frame_index=frame_index)
    assert np.array_equal(host(fr.counts), ref["alloc"].counts)
    for l in range(L):
        assert_rel(host(fr.layers[l]), ref["layers"][l], what=f"layer {l}")
    assert_rel(host(out), ref["hdr"], what="hdr")
    assert_rel(host(fr.ldr), ref["ldr"], atol=LDR_ATOL, what="ldr")
    return fr, ref


def test_frame_parity_128_plain(spp):
    """128 x 128, 0.25 spp, 2 levels, no temporal term (29 logits at full res)."""
    _frame_parity(spp, 128, 128, 2, 0.25, temporal=False)


def test_frame_parity_1080p_temporal(spp):
    """1920 x 1080, 0.25 spp, 3 levels, 54 logits, bilinear reprojection."""
    _frame_parity(spp, 1920, 1080, 3, 0.25, temporal=True)


def test_frame_parity_4k_low_budget(spp):
    """3840 x 2160 at 0.125 spp, 3 levels, temporal."""
    _frame_parity(spp, 3840, 2160, 3, 0.125, temporal=True, frame_index=2, seed=3)


def test_frame_parity_1440p_five_levels(spp):
    """The paper's five-level pyramid (Sec. 6.1, App. A) at 2560 x 1440 with
    the temporal term (1440 / 16 = 90, so every level is whole)."""
    _frame_parity(spp, 2560, 1440, 5, 0.25, temporal=True, frame_index=3, seed=4)


def test_two_frame_sequence_feeds_back(spp):
    """Frame t+1 reprojects frame t's HDR output (red loop of Sec. 3): each
    side feeds back its own output."""
    W, H, L, B = 256, 128, 3, 0.25
    fr = spp.Frame(W, H, L, max_budget=B)
    prev_gpu, prev_ref = None, None
    for t in range(2):
        x = inp.frame_inputs(W, H, L, frame=t, temporal=True)
        params = spp.make_params(B, frame=t)
        out = fr.run(dev(x["d"]), dev(x["clean"]), [dev(a) for a in x["logits"]], params,
                     prev=prev_gpu, mv=dev(x["mv"]), mask=dev(x["mask"]))
        ref = oracle.frame(x["d"], x["clean"], [a.astype(np.float64) for a in x["logits"]], W, H,
                           L, B, prev=prev_ref, mv=x["mv"], mask=x["mask"], frame_index=t)
        torch.cuda.synchronize()
        assert_rel(host(out), ref["hdr"], rtol=2e-5 if t else RTOL, what=f"frame {t}")
        prev_gpu, prev_ref = out, ref["hdr"]


def test_dependent_launch_gives_identical_frames(spp):
    """Programmatic dependent launch changes only when the kernels are
    scheduled: a sequence of frames run back to back (no host sync between
    kernels) is bit for bit the same with it on and off."""
    from paper_2602_08642_gb300 import _binding as Bnd
    W, H, L, B = 640, 360, 3, 0.25
    xs = [inp.frame_inputs(W, H, L, frame=t, temporal=True) for t in range(3)]
    xs = [dict(d=dev(x["d"]), clean=dev(x["clean"]), logits=[dev(a) for a in x["logits"]],
               mv=dev(x["mv"]), mask=dev(x["mask"])) for x in xs]
    outs = {}
    was = Bnd.spp_get_dependent_launch()
    try:
        for on in (True, False):
            Bnd.spp_set_dependent_launch(on)
            fr = spp.Frame(W, H, L, max_budget=B)
            fr.clear_status()
            prev, got = None, []
            for t, x in enumerate(xs):
                out = fr.run(x["d"], x["clean"], x["logits"], spp.make_params(B, frame=t),
                             prev=prev, mv=x["mv"], mask=x["mask"])
                got.append((fr.counts.clone(), out.clone(), fr.ldr.clone()))
                prev = out
            torch.cuda.synchronize()
            assert fr.check_status() == 0
            outs[on] = got
    finally:
        Bnd.spp_set_dependent_launch(was)
    for a, b in zip(outs[True], outs[False]):
        for u, v in zip(a, b):
            assert torch.equal(u, v)


# ---------------------------------------------------------------------------
# Blue-noise dithered discretisation (Sec. 6.3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("W,H,B,T", [(128, 128, 0.25, 64), (1000, 700, 0.37, 64),
                                     (97, 61, 1.6, 16), (1920, 1080, 0.25, 64)])
def test_alloc_dithered_bit_exact(spp, W, H, B, T):
    import oracle.bluenoise as BN
    d = inp.density_lognormal(W, H, seed=31)
    mask = spp.binding.spp_blue_noise_mask(T, 0xB1)
    params = spp.make_params(B, seed=0x5EED, frame=5)
    fr = spp.Frame(W, H, 2, max_budget=B)
    fr.clear_status()
    mdev = torch.from_numpy(mask.view(np.int16)).cuda()
    spp.check(spp.binding.spp_alloc_sample_map_dithered(
        dev(d), W, H, params, mdev, fr.counts, fr.offsets, fr.sample_pixel, fr.capacity, fr.s,
        fr.holdout_w, fr.total, fr.status, fr.alloc_ws))
    torch.cuda.synchronize()
    assert fr.check_status() == 0
    u48 = BN.uniform48(BN.mask(T, 0xB1), W, H, seed=0x5EED, frame=5)
    ref = oracle.alloc(d, B, u48=u48)
    assert np.array_equal(host(fr.counts), ref.counts)
    assert np.array_equal(host(fr.offsets)[:W * H + 1], ref.offsets)
    assert int(fr.total.item()) == ref.T


def test_alloc_dithered_constant_density_budget(spp):
    """A constant density over whole tiles receives its budget to within one
    sample per tile, frame after frame (white noise: hundreds off)."""
    import oracle.bluenoise as BN
    W = H = 256
    T = 64
    mask = torch.from_numpy(spp.binding.spp_blue_noise_mask(T, 3).view(np.int16)).cuda()
    d = torch.ones(H, W, device="cuda")
    fr = spp.Frame(W, H, 2, max_budget=0.5)
    for frame in range(6):
        params = spp.make_params(0.3, frame=frame)
        spp.check(spp.binding.spp_alloc_sample_map_dithered(
            d, W, H, params, mask, fr.counts, fr.offsets, fr.sample_pixel, fr.capacity, fr.s,
            fr.holdout_w, fr.total, fr.status, fr.alloc_ws))
        assert abs(int(fr.total.item()) - 0.3 * W * H) <= (W // T) * (H // T)
