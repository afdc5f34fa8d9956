"""Seeded synthetic inputs shaped like the paper's workloads.

A module of its own: the CUDA path and the FP64 oracle both read their inputs
from here, and it imports neither of them.

This module holds none of the method's arithmetic: it only draws the inputs
(sampler density, clean procedural scene, G-buffer, kernel logits, motion
vectors, disocclusion masks) that both the CUDA path and the FP64 oracle
consume.  They stand in for the paper's Falcor renders of the extended
Noisebase dataset, which are not available here.

Recipe (all numpy, seeded per call):
  density   d = exp(sigma Z), Z ~ N(0,1) i.i.d., sigma = 1   (FP32 [H][W])
  scene     albedo from 16 seeded half-planes and discs painted over a
            background (piecewise constant, in [0.05, 1]), times a smooth
            illumination made of 3 seeded low-frequency sinusoids per
            channel; clipped to RGB in [0, 4]                  (FP32 [3][H][W])
  G-buffer  albedo (above), unit normals of a smooth seeded height field,
            depth in [1, 100], piecewise smooth with the same edges
  logits    N(0,1) i.i.d. per channel and level: 54 / 29 / 25 channels at
            full / intermediate / coarsest resolution (29 at full resolution
            when there is no temporal term)
  fixed     the plain fixed-kernel reconstruction: denoise tap (i,j) gets
            -(i^2+j^2)/2, upsampling and temporal taps 0
  motion    affine field mv = A (p - c) + b in pixels, |mv| <= 8 px
  mask      seeded discs covering ~5% of the pixels (uint8, 1 = disoccluded)
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed) & 0xFFFFFFFF, *stream]))


def density_lognormal(W: int, H: int, seed: int = 1, sigma: float = 1.0) -> np.ndarray:
    z = _rng(seed, 11).standard_normal((H, W), dtype=np.float32)
    return np.exp(np.float32(sigma) * z).astype(np.float32)


def _shapes(W: int, H: int, seed: int, frame: int, count: int = 16):
    """Label map of painted half-planes / discs and their per-shape values."""
    r = _rng(seed, 21)
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float32)
    # the whole scene drifts a little per frame so that frames are related
    dx, dy = 1.5 * frame, -0.75 * frame
    xs = xs - dx
    ys = ys - dy
    label = np.zeros((H, W), np.int16)
    scale = float(max(W, H))
    for k in range(1, count + 1):
        if r.random() < 0.5:  # half-plane through a random point
            px, py = r.random() * W, r.random() * H
            th = r.random() * 2 * np.pi
            inside = (np.cos(th) * (xs - px) + np.sin(th) * (ys - py)) > 0
        else:
            cx, cy = r.random() * W, r.random() * H
            rad = (0.05 + 0.2 * r.random()) * scale
            inside = (xs - cx) ** 2 + (ys - cy) ** 2 < rad * rad
        label[inside] = k
    albedo = r.uniform(0.05, 1.0, size=(count + 1, 3)).astype(np.float32)
    depth_base = r.uniform(1.0, 60.0, size=count + 1).astype(np.float32)
    return label, albedo, depth_base, xs, ys


def scene(W: int, H: int, seed: int = 3, frame: int = 0):
    """Clean image [3][H][W] in [0,4] plus G-buffer dict (albedo, normal, depth)."""
    label, albedo_tab, depth_tab, xs, ys = _shapes(W, H, seed, frame)
    r = _rng(seed, 31)
    albedo = np.transpose(albedo_tab[label], (2, 0, 1))  # [3][H][W]
    illum = np.empty((3, H, W), np.float32)
    u = xs / max(W, 1)
    v = ys / max(H, 1)
    for c in range(3):
        acc = np.full((H, W), 1.0, np.float32)
        for _ in range(3):
            fx, fy = r.uniform(0.5, 4.0, size=2)
            ph = r.uniform(0, 2 * np.pi)
            amp = r.uniform(0.15, 0.35)
            acc += np.float32(amp) * np.sin(2 * np.pi * (fx * u + fy * v) + ph).astype(np.float32)
        illum[c] = acc
    clean = np.ascontiguousarray(np.clip(2.2 * albedo * illum, 0.0, 4.0), dtype=np.float32)
    # height field for normals: smooth bumps
    hgt = np.zeros((H, W), np.float32)
    for _ in range(3):
        fx, fy = r.uniform(0.5, 3.0, size=2)
        ph = r.uniform(0, 2 * np.pi)
        hgt += np.sin(2 * np.pi * (fx * u + fy * v) + ph).astype(np.float32)
    gy, gx = np.gradient(hgt * 0.05 * max(W, H))
    nrm = np.stack([-gx, -gy, np.ones_like(gx)])
    nrm /= np.linalg.norm(nrm, axis=0, keepdims=True)
    depth = depth_tab[label] + 0.3 * hgt + 0.002 * (xs + ys)
    depth = np.clip(depth, 1.0, 100.0).astype(np.float32)
    gbuf = dict(albedo=np.ascontiguousarray(albedo, dtype=np.float32),
                normal=np.ascontiguousarray(nrm, dtype=np.float32),
                depth=np.ascontiguousarray(depth[None], dtype=np.float32))
    return clean, gbuf


def logit_channels(level: int, L: int, temporal: bool) -> int:
    if level == L - 1:
        return 25
    if level == 0 and temporal:
        return 54
    return 29


def random_logits(W: int, H: int, L: int, seed: int = 2, temporal: bool = True,
                  scale: float = 1.0) -> list[np.ndarray]:
    r = _rng(seed, 41)
    out = []
    for l in range(L):
        C = logit_channels(l, L, temporal)
        z = r.standard_normal((C, H >> l, W >> l), dtype=np.float32)
        if scale != 1.0:
            z *= np.float32(scale)
        out.append(z)
    return out


def fixed_logits(W: int, H: int, L: int, temporal: bool = True) -> list[np.ndarray]:
    """Plain fixed-kernel reconstruction: Gaussian-like denoise taps
    exp(-(i^2+j^2)/2) (as logits), flat upsampling and temporal taps."""
    out = []
    for l in range(L):
        C = logit_channels(l, L, temporal)
        vals = np.zeros(C, np.float32)
        for j in range(-2, 3):
            for i in range(-2, 3):
                vals[(j + 2) * 5 + (i + 2)] = -(i * i + j * j) / 2.0
        out.append(np.ascontiguousarray(
            np.broadcast_to(vals[:, None, None], (C, H >> l, W >> l)), dtype=np.float32))
    return out


def motion_affine(W: int, H: int, seed: int = 4, frame: int = 0, max_px: float = 8.0) -> np.ndarray:
    r = _rng(seed, 51, frame)
    A = r.uniform(-1.0, 1.0, size=(2, 2)) * (4.0 / max(W, H))
    b = r.uniform(-4.0, 4.0, size=2)
    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    mx = A[0, 0] * (xs - cx) + A[0, 1] * (ys - cy) + b[0]
    my = A[1, 0] * (xs - cx) + A[1, 1] * (ys - cy) + b[1]
    mag = np.sqrt(mx * mx + my * my).max() if W * H else 0.0
    if mag > max_px:
        mx *= max_px / mag
        my *= max_px / mag
    return np.stack([mx, my]).astype(np.float32)


def disocclusion_mask(W: int, H: int, seed: int = 5, frame: int = 0, frac: float = 0.05,
                      discs: int = 24) -> np.ndarray:
    r = _rng(seed, 61, frame)
    m = np.zeros((H, W), np.uint8)
    if W * H == 0 or frac <= 0:
        return m
    rad = np.sqrt(frac * W * H / (np.pi * discs))
    target = int(frac * W * H)
    covered = 0
    for _ in range(discs * 8):
        cx, cy = r.random() * W, r.random() * H
        rr = rad * r.uniform(0.5, 1.5)
        x0, x1 = max(int(cx - rr), 0), min(int(cx + rr) + 1, W)
        y0, y1 = max(int(cy - rr), 0), min(int(cy + rr) + 1, H)
        if x0 >= x1 or y0 >= y1:
            continue
        yy, xx = np.mgrid[y0:y1, x0:x1]
        box = m[y0:y1, x0:x1]
        before = int(box.sum())
        box |= (((xx - cx) ** 2 + (yy - cy) ** 2) < rr * rr).astype(np.uint8)
        covered += int(box.sum()) - before
        if covered >= target:
            break
    return m


def frame_inputs(W: int, H: int, L: int, frame: int, *, temporal: bool = True,
                 base_seed: int = 1, fixed: bool = False) -> dict:
    """All per-frame inputs of the plain method for frame ``frame``."""
    d = density_lognormal(W, H, seed=base_seed * 1000 + frame)
    clean, gbuf = scene(W, H, seed=base_seed * 1000 + 300, frame=frame)
    lg = (fixed_logits(W, H, L, temporal) if fixed
          else random_logits(W, H, L, seed=base_seed * 1000 + 100 + frame, temporal=temporal))
    mv = motion_affine(W, H, seed=base_seed * 1000 + 400, frame=frame)
    mask = disocclusion_mask(W, H, seed=base_seed * 1000 + 500, frame=frame)
    return dict(d=d, clean=clean, gbuf=gbuf, logits=lg, mv=mv, mask=mask)


def unet_params(layers, seed: int = 7, head_bias: dict | None = None,
                head_scale: float = 0.01) -> np.ndarray:
    """Flat FP32 parameter vector for a stack of 3x3 convolutions.

    ``layers`` is a list of (name, cin, cout, relu); for each layer the
    weights [cout][cin][3][3] (He-normal, std sqrt(2 / (9 cin)); heads, the
    layers without ReLU, scaled by ``head_scale``) are followed by the bias
    [cout] (zero, or ``head_bias[name]`` for a head)."""
    r = _rng(seed, 71)
    parts = []
    for name, cin, cout, relu in layers:
        w = r.standard_normal((cout, cin, 3, 3)) * np.sqrt(2.0 / (9 * cin))
        if not relu:
            w *= head_scale
        b = np.zeros(cout)
        if head_bias is not None and name in head_bias:
            b[:] = head_bias[name]
        parts += [w.ravel(), b]
    return np.concatenate(parts).astype(np.float32)


def fixed_head_bias() -> dict:
    """Head biases that make a network with near-zero head weights start as
    the plain fixed-kernel method (the values of :func:`fixed_logits`, zero
    density logit)."""
    g = np.zeros(25, np.float32)
    for j in range(-2, 3):
        for i in range(-2, 3):
            g[(j + 2) * 5 + (i + 2)] = -(i * i + j * j) / 2.0
    h0 = np.zeros(55, np.float32)
    h0[:25] = g
    h1 = np.zeros(29, np.float32)
    h1[:25] = g
    return {"h0": h0, "h1": h1, "h2": g.copy()}


def scene_motion(W: int, H: int, frame: int = 1) -> np.ndarray:
    """Motion vectors (current -> previous frame, pixels) of :func:`scene`,
    whose content drifts by (+1.5, -0.75) px per frame: the constant field
    (-1.5, +0.75)."""
    mv = np.empty((2, H, W), np.float32)
    mv[0] = -1.5
    mv[1] = 0.75
    return mv


def training_pair(size: int, seed: int, frame: int = 1):
    """Two consecutive frames of one procedural scene at size x size: dict
    with clean / gbuf of frames t-1 and t and the true motion of frame t."""
    c0, g0 = scene(size, size, seed=seed, frame=frame - 1)
    c1, g1 = scene(size, size, seed=seed, frame=frame)
    return dict(clean_prev=c0, gbuf_prev=g0, clean=c1, gbuf=g1, mv=scene_motion(size, size, frame))
