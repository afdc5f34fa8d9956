"""FP64 oracle of the learned predictor (the sampler / kernel network of
Sec. 3 and Sec. 6.3) and of its backward.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests,
``__graft_entry__.smoke()`` and the CPU baseline leg of ``bench.py`` call it;
the product never imports it, and it imports nothing from the product.

The paper trains a U-Net that maps G-buffers (and the previous output) to
the sampling density and to the per-pixel kernel logits of every pyramid
level (Sec. 3, Sec. 6.3, Appendix A).  It does not print the layer table;
the network here is the reading used throughout this repository:

    features (12 ch, full resolution)
      e0a 12->32, e0b 32->32                        -> s0   (level 0)
      avg-pool 2x2, e1a 32->64, e1b 64->64          -> s1   (level 1)
      avg-pool 2x2, e2a 64->128, e2b 128->128       -> b    (level 2)
      h2  128->25                                   -> logits of level 2
      nearest-upsample b, concat [s1, up b] (192),
      d1a 192->64, d1b 64->64                       -> t1   (level 1)
      h1  64->29                                    -> logits of level 1
      nearest-upsample t1, concat [s0, up t1] (96),
      d0a 96->32, d0b 32->32                        -> t0   (level 0)
      h0  32->55  -> 54 logits of level 0 (kd 25, ku 4, kt 25) and the
                     density logit z (channel 54)

Every layer is a 3x3 convolution with zero padding and a bias; hidden layers
are followed by ReLU, heads are linear.  The density is the spatial softmax
of z (Sec. 3): d = exp(z - max z), normalised to the budget by the
allocation step.  Input features (Sec. 6.3 lists albedo, normal, depth and
motion; the previous output is the recurrent input of Sec. 3):
albedo (3), normal (3), ln(depth)/ln(100) (1), motion / 8 px (2), previous
LDR output warped to the current frame (3).

Parameters are one flat FP32 vector theta: for each layer in the order of
LAYERS, the weights [cout][cin][3][3] followed by the bias [cout].

Precision model of the GPU path (``round_bf16=True`` replays it): the input
features, the weights and every hidden activation (after ReLU, and after
each 2x2 average pool) are rounded to BF16 (round to nearest even, from the
FP32 value); sums and the heads stay in higher precision.  With
``round_bf16=False`` everything is exact FP64 (the error reference).

Pins (tests/test_oracle_unet_pins.py): the convolution against
scipy.signal.correlate2d; one-hot weights give a shifted copy; a
channel-copy network reduces to a closed form of pools and upsamples that
fixes the wiring (concat order, which level each head reads); the backward
against central finite differences; AdamW against its closed form on the
first step.
"""
from __future__ import annotations

import math

import numpy as np

# Network specifications: input channels and the output channels of the
# three heads (h0 at level 0, h1 at level 1, h2 at level 2; 0 = absent).
#   joint     the single predictor of density and kernels (12 inputs; h0 =
#             54 logits + density logit)
#   sampler   the first stage of the two-stage pipeline (Sec. 3): G-buffer,
#             warped previous output and warped latents -> density logit
#   denoiser  the second stage: noisy radiance, s and n, G-buffer, warped
#             previous HDR output and latents -> 54 logits, 3 demodulation
#             channels (Sec. 6.2) and 7 latent channels at level 0; 29 and 25
#             logits at levels 1 and 2
N_LATENT = 7
SPECS = {
    "joint": (12, (55, 29, 25)),
    "sampler": (12 + N_LATENT, (1, 0, 0)),
    "denoiser": (17 + N_LATENT, (64, 29, 25)),
}
DEMOD_CHANNELS = slice(54, 57)
LATENT_CHANNELS = slice(57, 57 + N_LATENT)
DEMOD_CLAMP = 8.0


def layers(spec: str = "joint"):
    """[(name, cin, cout, relu)] of a network specification (absent heads
    are left out; the order is the parameter order)."""
    cin, (c0, c1, c2) = SPECS[spec]
    out = [("e0a", cin, 32, True), ("e0b", 32, 32, True),
           ("e1a", 32, 64, True), ("e1b", 64, 64, True),
           ("e2a", 64, 128, True), ("e2b", 128, 128, True)]
    if c2:
        out.append(("h2", 128, c2, False))
    out += [("d1a", 192, 64, True), ("d1b", 64, 64, True)]
    if c1:
        out.append(("h1", 64, c1, False))
    out += [("d0a", 96, 32, True), ("d0b", 32, 32, True), ("h0", 32, c0, False)]
    return out


LAYERS = layers("joint")
N_FEATURES = 12
DENSITY_CHANNEL = 54


def param_offsets(spec: str = "joint"):
    """[(name, cin, cout, w_offset, b_offset)], total parameter count."""
    out, off = [], 0
    for name, cin, cout, _ in layers(spec):
        out.append((name, cin, cout, off, off + cout * cin * 9))
        off += cout * cin * 9 + cout
    return out, off


def unpack(theta, spec: str = "joint"):
    """dict name -> (W [cout][cin][3][3] FP64, b [cout] FP64)."""
    theta = np.asarray(theta, np.float64)
    table, total = param_offsets(spec)
    assert theta.size == total
    return {name: (theta[wo:bo].reshape(cout, cin, 3, 3), theta[bo:bo + cout])
            for name, cin, cout, wo, bo in table}


def round_bf16(x):
    """Round to BF16 (nearest, ties to even) from the FP32 value, returned as FP64."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


# --------------------------------------------------------------- features
def features(albedo, normal, depth, mv, prev_ldr):
    """[12][H][W] network input (Sec. 6.3 inputs plus the previous output)."""
    depth = np.asarray(depth, np.float64).reshape((1,) + np.shape(depth)[-2:])
    return np.concatenate([
        np.asarray(albedo, np.float64), np.asarray(normal, np.float64),
        np.log(depth) / math.log(100.0),
        np.asarray(mv, np.float64) / 8.0,
        np.asarray(prev_ldr, np.float64)])


# ------------------------------------------------------------ primitives
def conv3x3(x, w, b):
    """y[o][y][x] = b[o] + sum_{i,dy,dx} w[o][i][dy][dx] x[i][y+dy-1][x+dx-1],
    zero outside the image.  Written as the nine shifted tap products, each
    a matrix product over the input channels (np.tensordot, FP64)."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    y = np.broadcast_to(np.asarray(b, np.float64)[:, None, None], (w.shape[0], H, W)).copy()
    for dy in range(3):
        for dx in range(3):
            y += np.tensordot(w[:, :, dy, dx], xp[:, dy:dy + H, dx:dx + W], axes=1)
    return y


def conv3x3_backward(x, w, g):
    """(dL/dx, dL/dw, dL/db) of sum(g * conv3x3(x, w, b))."""
    C, H, W = x.shape
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    gxp = np.zeros_like(xp)
    gw = np.empty_like(w)
    for dy in range(3):
        for dx in range(3):
            gw[:, :, dy, dx] = np.tensordot(g, xp[:, dy:dy + H, dx:dx + W], axes=([1, 2], [1, 2]))
            gxp[:, dy:dy + H, dx:dx + W] += np.tensordot(w[:, :, dy, dx].T, g, axes=1)
    return gxp[:, 1:-1, 1:-1], gw, g.sum(axis=(1, 2))


def pool2(x):
    """2x2 average pool (the pyramid's box filter, Eq. app-pyramid)."""
    C, H, W = x.shape
    return x.reshape(C, H // 2, 2, W // 2, 2).mean(axis=(2, 4))


def pool2_backward(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def up2(x):
    """Nearest-neighbour x2 upsampling."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(g):
    C, H, W = g.shape
    return g.reshape(C, H // 2, 2, W // 2, 2).sum(axis=(2, 4))


# ---------------------------------------------------------------- network
def forward(theta, x, round_bf16_acts: bool = False, spec: str = "joint"):
    """Forward pass on one image x [cin][H][W] (H, W divisible by 4).

    Returns a dict with heads [h0 [c0][H][W], h1 [c1][H/2][W/2] or None,
    h2 [c2][H/4][W/4] or None] and the cache needed by :func:`backward`;
    for the joint network also z [H][W] and logits [l0 [54][H][W], l1, l2]."""
    P = unpack(theta, spec)
    rnd = round_bf16 if round_bf16_acts else (lambda a: a)
    if round_bf16_acts:
        P = {k: (round_bf16(w), b) for k, (w, b) in P.items()}
    cache = {}

    def layer(name, inp, relu=True):
        w, b = P[name]
        cache[name + ".in"] = inp
        y = conv3x3(inp, w, b)
        if relu:
            y = rnd(np.maximum(y, 0.0))
        cache[name + ".out"] = y
        return y

    x = rnd(np.asarray(x, np.float64))
    assert x.shape[0] == SPECS[spec][0]
    s0 = layer("e0b", layer("e0a", x))
    s1 = layer("e1b", layer("e1a", rnd(pool2(s0))))
    bt = layer("e2b", layer("e2a", rnd(pool2(s1))))
    l2 = layer("h2", bt, relu=False) if "h2" in P else None
    t1 = layer("d1b", layer("d1a", np.concatenate([s1, up2(bt)])))
    l1 = layer("h1", t1, relu=False) if "h1" in P else None
    t0 = layer("d0b", layer("d0a", np.concatenate([s0, up2(t1)])))
    h0 = layer("h0", t0, relu=False)
    out = dict(heads=[h0, l1, l2], cache=cache, params=P, spec=spec)
    if spec == "joint":
        out.update(z=h0[DENSITY_CHANNEL], logits=[h0[:DENSITY_CHANNEL], l1, l2])
    return out


def backward_heads(fwd, g_heads, input_grad: bool = False):
    """Gradient of sum_k <g_heads[k], heads[k]> with respect to theta (flat,
    the layout of :func:`param_offsets`), in FP64; with input_grad also the
    gradient with respect to the input x (returned as (g_theta, g_x))."""
    P, cache, spec = fwd["params"], fwd["cache"], fwd["spec"]
    grads = {}

    def back(name, g_out, relu=True):
        if relu:
            g_out = g_out * (cache[name + ".out"] > 0)
        gx, gw, gb = conv3x3_backward(cache[name + ".in"], P[name][0], g_out)
        grads[name] = (gw, gb)
        return gx

    g_t0 = back("h0", np.asarray(g_heads[0], np.float64), relu=False)
    g_cat0 = back("d0a", back("d0b", g_t0))
    c_s0 = cache["e0b.out"].shape[0]
    g_s0 = g_cat0[:c_s0]
    g_t1 = up2_backward(g_cat0[c_s0:])
    if "h1" in P:
        g_t1 = g_t1 + back("h1", np.asarray(g_heads[1], np.float64), relu=False)
    g_cat1 = back("d1a", back("d1b", g_t1))
    c_s1 = cache["e1b.out"].shape[0]
    g_s1 = g_cat1[:c_s1]
    g_b = up2_backward(g_cat1[c_s1:])
    if "h2" in P:
        g_b = g_b + back("h2", np.asarray(g_heads[2], np.float64), relu=False)
    g_s1 = g_s1 + pool2_backward(back("e2a", back("e2b", g_b)))
    g_s0 = g_s0 + pool2_backward(back("e1a", back("e1b", g_s1)))
    g_x = back("e0a", back("e0b", g_s0))
    table, total = param_offsets(spec)
    out = np.empty(total)
    for name, cin, cout, wo, bo in table:
        gw, gb = grads[name]
        out[wo:bo] = gw.ravel()
        out[bo:bo + cout] = gb
    return (out, g_x) if input_grad else out


def backward(fwd, g_logits, g_z):
    """Joint network: gradient of sum_l <g_logits[l], logits[l]> + <g_z, z>
    with respect to theta."""
    g_h0 = np.concatenate([np.asarray(g_logits[0], np.float64),
                           np.asarray(g_z, np.float64)[None]])
    return backward_heads(fwd, [g_h0, g_logits[1], g_logits[2]])


def density(z):
    """Unnormalised spatial softmax of the density logit (Sec. 3)."""
    z = np.asarray(z, np.float64)
    return np.exp(z - z.max())


# --------------------------------------------------------------- optimiser
def adamw(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step (Loshchilov & Hutter, decoupled weight decay), step t >= 1:
    m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
    theta -= lr (m/(1-b1^t) / (sqrt(v/(1-b2^t)) + eps) + wd theta)."""
    theta = np.asarray(theta, np.float64)
    g = np.asarray(g, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * (mh / (np.sqrt(vh) + eps) + wd * theta), m, v
