"""Parity of the predictor's training kernels (a11) with the FP64 oracle:
the tensor-core weight gradient, the whole network backward and AdamW.

Tolerances
* Weight gradient of one layer: the GPU sums BF16 products in FP32 over
  the pixels (MMA blocks of 16, then chunk after chunk in TMEM, then the
  splits in a fixed order); the error is bounded by a few times
  (pixels/16 + 64) * 2^-24 * sum |x g|.
* Network backward: the gradients between layers are stored in BF16 and
  the forward activations differ from the oracle's at the BF16 error level
  (see test_gpu_unet.py); per layer the relative L2 error of the weight and
  bias gradients is held below 5 %.
* AdamW: FP32 arithmetic against FP64 on the same FP32 hyper-parameters:
  parameters to 1e-5 relative, moments within a few FP32 roundings of
  their terms.
"""
import numpy as np
import pytest
import torch

import oracle.unet as U
import spp_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spp():
    from conftest import build_spp_lib
    build_spp_lib()
    import paper_2602_08642_gb300 as spp
    torch.cuda.set_device(0)
    return spp


def _nchw(t_nhwc):
    return t_nhwc.float().cpu().numpy().astype(np.float64).transpose(0, 3, 1, 2)


@pytest.mark.parametrize("cin,cout,B,H,W", [
    (32, 32, 2, 8, 200), (16, 64, 1, 6, 70), (64, 128, 1, 5, 129), (192, 64, 1, 4, 64),
    (96, 32, 2, 4, 33), (8, 32, 1, 3, 10), (128, 128, 1, 4, 300), (32, 56, 1, 2, 65)])
def test_conv3x3_backward_weights_parity(spp, cin, cout, B, H, W):
    g = torch.Generator().manual_seed(cin * 31 + cout + W)
    x = torch.randn(B, H, W, cin, generator=g).to(torch.bfloat16)
    gy = torch.randn(B, H, W, cout, generator=g).to(torch.bfloat16)
    gw = torch.empty(cout, cin, 3, 3, device="cuda")
    gb = torch.empty(cout, device="cuda")
    ws = torch.empty(spp.binding.spp_conv3x3_backward_weights_workspace_bytes(B, W, H, cin, cout),
                     dtype=torch.uint8, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")[:1]
    spp.check(spp.binding.spp_conv3x3_backward_weights(x.cuda(), gy.cuda(), B, W, H, cin, cout,
                                                       gw, gb, ws, st))
    assert spp.binding.spp_get_status(st) == 0
    xb, gyb = _nchw(x), _nchw(gy)
    ref_w = np.zeros((cout, cin, 3, 3))
    ref_b = np.zeros(cout)
    abs_w = np.zeros((cout, cin, 3, 3))
    wdum = np.zeros((cout, cin, 3, 3))
    for b in range(B):
        _, rw, rb = U.conv3x3_backward(xb[b], wdum, gyb[b])
        _, aw, _ = U.conv3x3_backward(np.abs(xb[b]), wdum, np.abs(gyb[b]))
        ref_w += rw
        ref_b += rb
        abs_w += aw
    npix = B * H * W
    tol = 4 * (npix / 16 + 64) * 2.0 ** -24
    got_w = gw.cpu().numpy().astype(np.float64)
    got_b = gb.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got_w - ref_w) <= tol * abs_w + 1e-30), \
        float((np.abs(got_w - ref_w) / (abs_w + 1e-30)).max())
    abs_b = np.abs(gyb).sum(axis=(0, 2, 3))
    assert np.all(np.abs(got_b - ref_b) <= tol * abs_b + 1e-30)


def _wgrad_multistage_shape(cin, min_chunks_per_cta=12):
    """(B, H, W) for which every CTA of the weight gradient (grid: M tiles of
    128 rows x pixel splits, one split per SM / M tiles) runs at least
    min_chunks_per_cta K chunks of 64 pixels, so that its 4 stages are
    reused three times over: W = 200 (three full chunks and a ragged one per
    row)."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cin_pad = (cin + 15) // 16 * 16
    mtiles = (9 * cin_pad + 127) // 128
    splits = max(1, sms // mtiles)
    H = int(np.ceil(min_chunks_per_cta * splits / 4))
    return 1, H, 200


@pytest.mark.parametrize("cin,cout", [(32, 32), (96, 32), (64, 128), (192, 64), (128, 128),
                                      (16, 64)])
def test_conv3x3_backward_weights_parity_multistage(spp, cin, cout):
    B, H, W = _wgrad_multistage_shape(cin)
    test_conv3x3_backward_weights_parity(spp, cin, cout, B, H, W)


def test_adamw_parity(spp):
    rng = np.random.default_rng(3)
    n = 100_003
    th, g = rng.standard_normal(n), rng.standard_normal(n)
    m, v = 0.1 * rng.standard_normal(n), np.abs(rng.standard_normal(n)) * 0.01
    c = lambda a: torch.from_numpy(a.astype(np.float32)).cuda()
    tt, gg, mm, vv = c(th), c(g), c(m), c(v)
    spp.check(spp.binding.spp_adamw_step(tt, gg, mm, vv, 7, lr=2e-3, weight_decay=0.01,
                                         grad_scale=0.5))
    f32 = lambda a: np.asarray(a).astype(np.float32).astype(np.float64)
    # the kernel's hyper-parameters are FP32 (0.999 is not representable):
    # the oracle takes the same values
    hp = dict(lr=float(f32(2e-3)), b1=float(f32(0.9)), b2=float(f32(0.999)),
              eps=float(f32(1e-8)), wd=float(f32(0.01)))
    rt, rm, rv = U.adamw(f32(th), 0.5 * f32(g), f32(m), f32(v), 7, **hp)
    assert np.allclose(tt.cpu().numpy(), rt, rtol=1e-5, atol=1e-7)
    # the moments are sums of two FP32 products: within a few FP32 roundings
    # of the magnitudes of their terms (they may cancel)
    gs = 0.5 * f32(g)
    tol_m = 2.0 ** -21 * (np.abs(f32(m)) + 0.1 * np.abs(gs))
    tol_v = 2.0 ** -21 * (f32(v) + 0.001 * gs * gs)
    assert np.all(np.abs(mm.cpu().numpy() - rm) <= tol_m)
    assert np.all(np.abs(vv.cpu().numpy() - rv) <= tol_v)


def _theta():
    table, total = U.param_offsets()
    theta = inp.unet_params(U.LAYERS, seed=21, head_scale=1.0).astype(np.float64)
    rng = np.random.default_rng(22)
    for name, cin, cout, wo, bo in table:
        theta[bo:bo + cout] = 0.05 * rng.standard_normal(cout)
    return theta.astype(np.float32)


def _features(B, W, H, seed):
    xs = []
    for b in range(B):
        clean, gb = inp.scene(W, H, seed=seed + b)
        mv = inp.motion_affine(W, H, seed=seed + b)
        prev = np.clip(clean / 4.0, 0, 1).astype(np.float32)
        xs.append(U.features(gb["albedo"], gb["normal"], gb["depth"], mv, prev))
    return np.stack(xs)


@pytest.mark.parametrize("B,W,H", [(2, 48, 32), (1, 136, 16)])
def test_unet_backward_parity(spp, B, W, H):
    theta = _theta()
    x = _features(B, W, H, seed=40)
    rng = np.random.default_rng(41)
    g0 = rng.standard_normal((B, 55, H, W)).astype(np.float32)
    g1 = rng.standard_normal((B, 29, H // 2, W // 2)).astype(np.float32)
    g2 = rng.standard_normal((B, 25, H // 4, W // 4)).astype(np.float32)
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    packed = torch.empty(spp.binding.spp_unet_packed_bytes(True), dtype=torch.uint8, device="cuda")
    spp.check(spp.binding.spp_unet_pack(c(theta), True, packed))
    fws = torch.empty(spp.binding.spp_predict_workspace_bytes(B, W, H), dtype=torch.uint8,
                      device="cuda")
    bws = torch.empty(spp.binding.spp_unet_backward_workspace_bytes(B, W, H), dtype=torch.uint8,
                      device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")[:1]
    xin = c(x)
    d = torch.empty(B, H, W, device="cuda")
    l0 = torch.empty(B, 55, H, W, device="cuda")
    l1 = torch.empty(B, 29, H // 2, W // 2, device="cuda")
    l2 = torch.empty(B, 25, H // 4, W // 4, device="cuda")
    spp.check(spp.binding.spp_predict_density_and_kernels(packed, xin, B, W, H, d, l0, l1, l2,
                                                          fws, st))
    grad = torch.empty(theta.size, device="cuda")
    spp.check(spp.binding.spp_unet_backward(packed, xin, B, W, H, fws, c(g0), c(g1), c(g2), grad,
                                            bws, st))
    assert spp.binding.spp_get_status(st) == 0
    got = grad.cpu().numpy().astype(np.float64)
    ref = np.zeros(theta.size)
    for b in range(B):
        f = U.forward(theta, x[b], round_bf16_acts=True)
        ref += U.backward(f, [g0[b, :54], g1[b], g2[b]], g0[b, 54])
    table, _ = U.param_offsets()
    errs = {}
    for name, cin, cout, wo, bo in table:
        for part, sl in (("w", slice(wo, bo)), ("b", slice(bo, bo + cout))):
            e = np.linalg.norm(got[sl] - ref[sl]) / np.linalg.norm(ref[sl])
            errs[name + "." + part] = round(float(e), 5)
    print("relative L2 error of the parameter gradients:", errs)
    bad = {k: v for k, v in errs.items() if not v < 5e-2}
    assert not bad, bad
