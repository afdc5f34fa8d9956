"""FP64 oracle of the two-stage pipeline: a sampler network before rendering,
a denoiser network after it, shared recurrent latents and learned
demodulation (Sec. 3, Sec. 6.2 "Learned Demodulation", Sec. 6.3).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests,
``__graft_entry__.smoke()`` and the CPU baseline leg of ``bench.py`` call it;
the product never imports it.

The paper describes the pipeline without printing its layer tables or the
exact input encodings; the reading implemented here:

* sampler (network spec "sampler", oracle/unet.py): input = the 12 features
  of the joint predictor (albedo, normal, ln(depth)/ln 100, motion / 8, the
  previous tone-mapped output warped to frame t) followed by the 7 latent
  channels of frame t-1 warped to frame t; head h0 = the density logit z.
* denoiser (spec "denoiser"): input, in this order, ln(1 + L^0) (3, the
  noisy splatted radiance), ln(1 + s) (the continuous sample map), ln(1 + n)
  (the integer counts), albedo (3), normal (3), ln(depth)/ln 100, motion / 8
  (2), ln(1 + W_t L_{t-1}) (3, the previous HDR output warped to frame t) and
  the 7 warped latents = 24 channels.  Head h0 = 54 kernel logits (kd, ku,
  kt), 3 demodulation channels c and 7 latent channels; h1 = 29 and h2 = 25
  kernel logits.
* demodulation map m = exp(clamp(c, -8, 8)) per colour channel (positive,
  1 at c = 0); the latents passed to the next frame are tanh of their
  channels.
* reconstruction with demodulation: the noisy radiance and the warped
  previous output are divided by m, the pyramid (Eq. app-pyramid) is built
  from L^0 / m, the gather pyramid (Eqs. app-recon-*) runs unchanged, and its
  full-resolution result is multiplied by m (remodulation) before the tone
  map:  out = m * R(pyr(L^0 / m), W_t L_{t-1} / m, kernels).

Pins (tests/test_oracle_two_stage_pins.py): the pyramid equals the one the
splat oracle builds; m = 1 reduces to the plain reconstruction; a constant m
cancels exactly (the gathers are linear and their weights do not depend on
the radiance); the backward against central finite differences; the
network's input gradient against finite differences; the feature channel
layout against closed forms.
"""
from __future__ import annotations

import math

import numpy as np

import oracle
from . import unet as U

N_LATENT = U.N_LATENT
DEMOD_CLAMP = U.DEMOD_CLAMP


# ------------------------------------------------------------- features
def warp_channels(field, mv) -> np.ndarray:
    """Bilinear warp W_t (the same definition as the previous-frame warp of
    Appendix A) of every channel of field [C][H][W]."""
    field = np.asarray(field, np.float64)
    C = field.shape[0]
    pad = (-C) % 3
    f = np.concatenate([field, np.zeros((pad,) + field.shape[1:])]) if pad else field
    out = np.concatenate([oracle.warp(f[k:k + 3], mv) for k in range(0, f.shape[0], 3)])
    return out[:C]


def sampler_features(albedo, normal, depth, mv, warped_prev_ldr=None, warped_latent=None):
    """[12 + N_LATENT][H][W] input of the sampler network."""
    H, W = np.shape(depth)[-2:]
    prev = np.zeros((3, H, W)) if warped_prev_ldr is None else warped_prev_ldr
    lat = np.zeros((N_LATENT, H, W)) if warped_latent is None else warped_latent
    return np.concatenate([U.features(albedo, normal, depth, mv, prev),
                           np.asarray(lat, np.float64)])


def denoiser_features(L0, s, n, albedo, normal, depth, mv, warped_prev_hdr=None,
                      warped_latent=None):
    """[17 + N_LATENT][H][W] input of the denoiser network."""
    H, W = np.shape(depth)[-2:]
    prev = np.zeros((3, H, W)) if warped_prev_hdr is None else warped_prev_hdr
    lat = np.zeros((N_LATENT, H, W)) if warped_latent is None else warped_latent
    depth = np.asarray(depth, np.float64).reshape(1, H, W)
    return np.concatenate([
        np.log1p(np.asarray(L0, np.float64)),
        np.log1p(np.asarray(s, np.float64).reshape(1, H, W)),
        np.log1p(np.asarray(n, np.float64).reshape(1, H, W)),
        np.asarray(albedo, np.float64), np.asarray(normal, np.float64),
        np.log(depth) / math.log(100.0),
        np.asarray(mv, np.float64) / 8.0,
        np.log1p(np.asarray(prev, np.float64)),
        np.asarray(lat, np.float64)])


def denoiser_features_backward(L0, s, g_x):
    """(dLoss/dL^0, dLoss/ds) from the gradient g_x [24][H][W] with respect
    to the denoiser's input (the other channels do not depend on L^0, s)."""
    H, W = np.shape(L0)[-2:]
    g_L0 = g_x[0:3] / (1.0 + np.asarray(L0, np.float64))
    g_s = g_x[3] / (1.0 + np.asarray(s, np.float64).reshape(H, W))
    return g_L0, g_s


def demod_map(h0) -> np.ndarray:
    """m = exp(clamp(c, -8, 8)) from the denoiser's level-0 head."""
    return np.exp(np.clip(np.asarray(h0, np.float64)[U.DEMOD_CHANNELS], -DEMOD_CLAMP,
                          DEMOD_CLAMP))


def latent(h0) -> np.ndarray:
    """The latents passed to the next frame: tanh of the latent channels."""
    return np.tanh(np.asarray(h0, np.float64)[U.LATENT_CHANNELS])


# ------------------------------------------------------ demodulated frame
def pyramid(L0, L: int) -> list[np.ndarray]:
    """Eq. app-pyramid: level l is the mean over the 2^l x 2^l block."""
    L0 = np.asarray(L0, np.float64)
    C, H, W = L0.shape
    out = [L0]
    for l in range(1, L):
        f = 1 << l
        out.append(L0.reshape(C, H // f, f, W // f, f).mean(axis=(2, 4)))
    return out


def reconstruct_demod(L0, c, logits, warped=None, mask=None, L: int = 3):
    """Reconstruction with learned demodulation; c [3][H][W] are the raw
    demodulation channels, warped the previous HDR output already warped to
    frame t (or None: no temporal term).  Returns (hdr, cache)."""
    L0 = np.asarray(L0, np.float64)
    c = np.asarray(c, np.float64)
    m = np.exp(np.clip(c, -DEMOD_CLAMP, DEMOD_CLAMP))
    L0d = L0 / m
    Wd = None if warped is None else np.asarray(warped, np.float64) / m
    layers = pyramid(L0d, L)
    hats = [None] * L
    for l in range(L - 1, -1, -1):
        coarse = hats[l + 1] if l + 1 < L else None
        hats[l] = oracle.reconstruct_level(layers[l], logits[l], coarse,
                                           Wd if l == 0 else None, mask if l == 0 else None)
    hdr = m * hats[0]
    return hdr, dict(m=m, L0d=L0d, Wd=Wd, layers=layers, hats=hats, c=c)


def reconstruct_demod_backward(L0, c, logits, g_hdr, warped=None, mask=None, L: int = 3):
    """Gradients of <g_hdr, hdr> of :func:`reconstruct_demod`: returns
    (g_logits per level, g_L0, g_c)."""
    hdr, k = reconstruct_demod(L0, c, logits, warped, mask, L)
    m, layers, hats = k["m"], k["layers"], k["hats"]
    g = np.asarray(g_hdr, np.float64) * m  # through the remodulation
    g_logits, g_noisy = [None] * L, [None] * L
    g_Wd = None
    for l in range(L):
        coarse = hats[l + 1] if l + 1 < L else None
        gl, gn, gc, gw = oracle.reconstruct_level_backward(
            layers[l], logits[l], g, coarse, k["Wd"] if l == 0 else None,
            mask if l == 0 else None)
        g_logits[l], g_noisy[l] = gl, gn
        if l == 0:
            g_Wd = gw
        g = gc
    H, W = np.shape(L0)[-2:]
    g_L0d = oracle.pyramid_backward(g_noisy, W, H)
    # d/dm of m * R(L0 / m, W / m):  R g_hdr - g_L0d L0 / m^2 - g_Wd W / m^2,
    # times dm/dc = m inside the clamp
    g_mc = np.asarray(g_hdr, np.float64) * hdr - g_L0d * k["L0d"]
    if g_Wd is not None:
        g_mc = g_mc - g_Wd * k["Wd"]
    g_c = g_mc * (np.abs(k["c"]) < DEMOD_CLAMP)
    return g_logits, g_L0d / m, g_c
