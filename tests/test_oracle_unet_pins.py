"""Pins of the FP64 network oracle (oracle/unet.py) against things other
than itself: a library convolution, shifted copies, a closed form of the
wiring, finite differences, the AdamW closed form and a library BF16
conversion."""
import numpy as np
import pytest
import torch

import oracle.unet as U
import spp_inputs as inp

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv3x3_matches_scipy_correlate():
    """Eq. of a 3x3 'same' convolution with zero padding: the library's
    2-D cross-correlation summed over input channels plus the bias."""
    rng = np.random.default_rng(1)
    x = rng.standard_normal((5, 11, 7))
    w = rng.standard_normal((4, 5, 3, 3))
    b = rng.standard_normal(4)
    y = U.conv3x3(x, w, b)
    for o in range(4):
        ref = b[o] + sum(scipy_signal.correlate2d(x[i], w[o, i], mode="same", boundary="fill")
                         for i in range(5))
        assert np.allclose(y[o], ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("dy,dx", [(0, 0), (0, 2), (2, 1), (1, 1)])
def test_one_hot_weights_give_shifted_copy(dy, dx):
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 6, 9))
    w = np.zeros((2, 3, 3, 3))
    w[1, 2, dy, dx] = 1.0
    y = U.conv3x3(x, w, np.zeros(2))
    assert np.all(y[0] == 0)
    H, W = 6, 9
    ref = np.zeros((H, W))
    for yy in range(H):
        for xx in range(W):
            sy, sx = yy + dy - 1, xx + dx - 1
            if 0 <= sy < H and 0 <= sx < W:
                ref[yy, xx] = x[2, sy, sx]
    assert np.array_equal(y[1], ref)


def _block_mean(a, k):
    H, W = a.shape
    return a.reshape(H // k, k, W // k, k).mean(axis=(1, 3))


def _expand(a, k):
    return np.kron(a, np.ones((k, k)))


def test_channel_copy_network_closed_form():
    """Every hidden layer copies channel 0 through its centre tap; the two
    decoder convolutions add the skip's channel 0 and the upsampled
    channel 0 (channels 64 and 32 of the concatenations); every head
    channel reads channel 0.  For a non-negative input channel a the
    outputs are then
        level 2: A4 = block mean of a over 4x4
        level 1: A2 + expand(A4)            (A2: 2x2 block mean)
        level 0: a + expand(A2) + expand(A4)
    which fixes which tensor each concatenation, pool, upsample and head
    reads."""
    table, total = U.param_offsets()
    theta = np.zeros(total)
    for name, cin, cout, wo, bo in table:
        w = theta[wo:bo].reshape(cout, cin, 3, 3)
        if name.startswith("h"):
            w[:, 0, 1, 1] = 1.0
        else:
            w[0, 0, 1, 1] = 1.0
        if name == "d1a":
            w[0, 64, 1, 1] = 1.0
        if name == "d0a":
            w[0, 32, 1, 1] = 1.0
    rng = np.random.default_rng(3)
    x = rng.random((12, 16, 8))
    f = U.forward(theta, x)
    a = x[0]
    A2, A4 = _block_mean(a, 2), _block_mean(a, 4)
    l2 = A4
    l1 = A2 + _expand(A4, 2)
    l0 = a + _expand(A2, 2) + _expand(A4, 4)
    assert np.allclose(f["logits"][2], l2[None], atol=1e-12)
    assert np.allclose(f["logits"][1], l1[None], atol=1e-12)
    assert np.allclose(f["logits"][0], l0[None], atol=1e-12)
    assert np.allclose(f["z"], l0, atol=1e-12)


def test_pool_and_upsample_backward_are_transposes():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, 8, 6))
    g = rng.standard_normal((3, 4, 3))
    assert abs((U.pool2(x) * g).sum() - (x * U.pool2_backward(g)).sum()) < 1e-12
    y = rng.standard_normal((3, 4, 3))
    G = rng.standard_normal((3, 8, 6))
    assert abs((U.up2(y) * G).sum() - (y * U.up2_backward(G)).sum()) < 1e-12


def _fd_check(f, x, grad, idxs, eps=1e-6, rtol=1e-6, atol=1e-9):
    for i in idxs:
        xp = x.copy()
        xm = x.copy()
        xp.flat[i] += eps
        xm.flat[i] -= eps
        fd = (f(xp) - f(xm)) / (2 * eps)
        assert abs(fd - grad.flat[i]) <= rtol * max(abs(fd), abs(grad.flat[i])) + atol, \
            (int(i), fd, grad.flat[i])


def test_conv3x3_backward_matches_fd():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((3, 5, 6))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    g = rng.standard_normal((4, 5, 6))
    gx, gw, gb = U.conv3x3_backward(x, w, g)
    _fd_check(lambda v: (U.conv3x3(v, w, b) * g).sum(), x, gx, range(x.size))
    _fd_check(lambda v: (U.conv3x3(x, v, b) * g).sum(), w, gw, range(w.size))
    _fd_check(lambda v: (U.conv3x3(x, w, v) * g).sum(), b, gb, range(b.size))


def test_network_backward_matches_fd():
    """Central differences of <g, outputs> with respect to parameters drawn
    from every layer, on an 8 x 8 image (2 x 2 at level 2)."""
    rng = np.random.default_rng(6)
    theta = inp.unet_params(U.LAYERS, seed=11, head_scale=1.0).astype(np.float64)
    theta[:] += 0.05 * rng.standard_normal(theta.size)  # non-zero biases too
    x = rng.random((12, 8, 8))
    gl = [rng.standard_normal((54, 8, 8)), rng.standard_normal((29, 4, 4)),
          rng.standard_normal((25, 2, 2))]
    gz = rng.standard_normal((8, 8))

    def loss(th):
        f = U.forward(th, x)
        return (sum(float((a * b).sum()) for a, b in zip(f["logits"], gl))
                + float((f["z"] * gz).sum()))

    grad = U.backward(U.forward(theta, x), gl, gz)
    table, _ = U.param_offsets()
    idxs = []
    for name, cin, cout, wo, bo in table:
        idxs += list(rng.choice(np.arange(wo, bo), size=6, replace=False))
        idxs += list(rng.choice(np.arange(bo, bo + cout), size=2, replace=False))
    _fd_check(loss, theta, grad, idxs, eps=1e-6, rtol=1e-5, atol=1e-8)


def test_adamw_first_step_closed_form():
    """At t = 1 from zero moments the bias-corrected moments are g and g^2,
    so the step is lr (g / (|g| + eps) + wd theta)."""
    rng = np.random.default_rng(7)
    th = rng.standard_normal(100)
    g = rng.standard_normal(100)
    lr, eps, wd = 3e-3, 1e-8, 0.01
    new, m, v = U.adamw(th, g, np.zeros(100), np.zeros(100), 1, lr=lr, eps=eps, wd=wd)
    assert np.allclose(new, th - lr * (g / (np.abs(g) + eps) + wd * th), rtol=1e-12, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a zero gradient only decays the weights
    new0, _, _ = U.adamw(th, np.zeros(100), np.zeros(100), np.zeros(100), 1, lr=lr, wd=wd)
    assert np.allclose(new0, th * (1 - lr * wd), rtol=1e-14)


def test_round_bf16_matches_library_conversion():
    rng = np.random.default_rng(8)
    v = np.concatenate([rng.standard_normal(10000) * 10 ** rng.uniform(-6, 6, 10000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 65504.0]])
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(U.round_bf16(v), ref)


def test_rounded_forward_keeps_activations_in_bf16():
    rng = np.random.default_rng(9)
    theta = inp.unet_params(U.LAYERS, seed=3)
    f = U.forward(theta, rng.random((12, 8, 8)), round_bf16_acts=True)
    for k, a in f["cache"].items():
        if k.endswith(".out") and not k.startswith("h"):
            assert np.array_equal(U.round_bf16(a), a), k


def test_features_layout():
    H, W = 4, 6
    rng = np.random.default_rng(10)
    alb, nrm = rng.random((3, H, W)), rng.random((3, H, W))
    depth = np.full((1, H, W), 100.0)
    depth[0, 0, 0] = 1.0
    mv = np.full((2, H, W), 8.0)
    prev = rng.random((3, H, W))
    f = U.features(alb, nrm, depth, mv, prev)
    assert f.shape == (12, H, W)
    assert np.array_equal(f[:3], alb) and np.array_equal(f[3:6], nrm)
    assert f[6, 0, 0] == 0.0 and abs(f[6, 1, 1] - 1.0) < 1e-15
    assert np.all(f[7:9] == 1.0) and np.array_equal(f[9:], prev)


def test_conv_of_upsampled_input_is_four_phase_convolutions():
    """The decoder's upsampled half: a 3x3 convolution of a nearest-x2
    upsampled tensor equals, at output phase (a, b), a 2x2 convolution of the
    coarse tensor with merged taps (phase 0: taps 0 and +1 onto offset 0, tap
    -1 onto offset -1; phase 1: taps -1 and 0 onto offset 0, tap +1 onto
    offset +1), zero padding on both sides.  Checked in FP64 on random data,
    including the borders."""
    rng = np.random.default_rng(31)
    C, O, h, w = 3, 4, 5, 7
    x = rng.standard_normal((C, h, w))
    wt = rng.standard_normal((O, C, 3, 3))
    b = rng.standard_normal(O)
    full = U.conv3x3(U.up2(x), wt, b)
    xp = np.zeros((C, h + 2, w + 2))
    xp[:, 1:-1, 1:-1] = x
    # merged taps per phase and axis: offset (-1, 0, +1) -> which 3x3 taps
    merge = {0: {-1: [0], 0: [1, 2]}, 1: {0: [0, 1], 1: [2]}}
    for a in (0, 1):
        for c in (0, 1):
            out = np.broadcast_to(b[:, None, None], (O, h, w)).copy()
            for oy, tys in merge[a].items():
                for ox, txs in merge[c].items():
                    wm = sum(wt[:, :, ty, tx] for ty in tys for tx in txs)
                    out += np.einsum("oi,ihw->ohw", wm, xp[:, 1 + oy:1 + oy + h, 1 + ox:1 + ox + w])
            assert np.allclose(full[:, a::2, c::2], out, rtol=1e-12, atol=1e-12)
