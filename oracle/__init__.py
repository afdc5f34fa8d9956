"""FP64 CPU oracle for the sub-1-spp sampling and reconstruction path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path (the CUDA
library in ``paper_2602_08642_gb300``) never imports this package, and this
package imports nothing from the product.

The arithmetic lives in ``spp_oracle.c`` (plain C, FP64, no fused multiply-add);
this module compiles it with gcc and wraps each function with numpy arrays.
Each wrapper names the passage of arXiv 2602.08642 it follows.

Parity status per function (the pins live in ``tests/test_oracle_pins.py``):
all functions here are pinned by closed forms, invariants, library routines or
brute force; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spp_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
ERR_ARG = -1
ERR_INPUT = -2


def build(force: bool = False) -> str:
    """Compile ``spp_oracle.c`` into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    # OpenMP over pixels / rows when the compiler has it (results do not
    # depend on the thread count); one thread otherwise
    if subprocess.run(cmd[:-1] + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_U32 = ctypes.c_uint32
_D = ctypes.c_double
_I = ctypes.c_int


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "orc_set_threads": (None, [_I]),
            "orc_get_threads": (_I, []),
            "orc_splitmix64_mix": (_U64, [_U64]),
            "orc_splitmix64_next": (_U64, [_P]),
            "orc_pixel_bits": (_U64, [_U64, _U32, _U64]),
            "orc_pixel_uniform": (_D, [_U64, _U32, _U64]),
            "orc_exact_sum_f32": (_D, [_P, _I64]),
            "orc_exact_sum_f64": (_D, [_P, _I64]),
            "orc_budget_coeffs": (_I, [_P, _I64, _D, _D, _P, _P, _P]),
            "orc_assign_one": (None, [_D, _D, _D, _I, _P, _P, _P]),
            "orc_alloc": (_I, [_P, _I64, _D, _D, _D, _I, _U64, _U32, _P, _P, _P, _P, _P, _P]),
            "orc_alloc_u48": (_I, [_P, _I64, _D, _D, _D, _I, _P, _P, _P, _P, _P, _P, _P]),
            "orc_sample_list": (None, [_P, _I64, _P]),
            "orc_sample_noise": (_D, [_U64, _U32, _U64, _U64]),
            "orc_render": (None, [_P, _P, _I64, _U64, _U32, _P]),
            "orc_splat": (_I, [_P, _P, _P, _P, _P, _I, _I, _I, _P]),
            "orc_warp": (None, [_P, _P, _I, _I, _P]),
            "orc_reconstruct_level": (_I, [_P, _P, _I, _P, _P, _P, _I, _I, _P]),
            "orc_tau": (_D, [_D, _D, _D]),
            "orc_srgb_encode": (_D, [_D]),
            "orc_tonemap": (None, [_P, _I64, _D, _D, _D, _D, _D, _P]),
            "orc_reconstruct_level_backward": (_I, [_P, _P, _I, _P, _P, _P, _I, _I, _P, _P, _P,
                                                    _P, _P]),
            "orc_warp_backward": (None, [_P, _I, _I, _P, _P]),
            "orc_tonemap_backward": (None, [_P, _I64, _D, _D, _D, _D, _D, _P, _P]),
            "orc_l1_loss": (_D, [_P, _P, _I64, _P]),
            "orc_pyramid_backward": (None, [_P, _I, _I, _I, _P]),
            "orc_splat_backward": (None, [_P, _P, _P, _P, _I64, _D, _I, _U64, _U32, _P, _P, _P]),
            "orc_density_backward": (None, [_P, _I64, _D, _D, _P, _P]),
            "orc_density_forward": (None, [_P, _I64, _D, _D, _P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (n <= 0: all cores)."""
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# Counter-based generator (SplitMix64, Steele, Lea & Flood 2014)
# --------------------------------------------------------------------------
def splitmix64_mix(z: int) -> int:
    return int(_load().orc_splitmix64_mix(z & 0xFFFFFFFFFFFFFFFF))


def splitmix64_sequence(seed: int, count: int) -> list[int]:
    st = ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF)
    lib = _load()
    return [int(lib.orc_splitmix64_next(ctypes.byref(st))) for _ in range(count)]


def pixel_uniform(seed: int, frame: int, i: int) -> float:
    """u_i of Sec. 4.2 for pixel i of frame ``frame``."""
    return float(_load().orc_pixel_uniform(seed, frame, i))


# --------------------------------------------------------------------------
# a1: exact sum and budget normalisation (Sec. 3)
# --------------------------------------------------------------------------
def exact_sum_f32(v) -> float:
    v = _c(v, np.float32).ravel()
    return float(_load().orc_exact_sum_f32(_ptr(v), v.size))


def exact_sum_f64(v) -> float:
    v = _c(v, np.float64).ravel()
    return float(_load().orc_exact_sum_f64(_ptr(v), v.size))


def budget_coeffs(d, B: float, phi: float = 0.125):
    """(rc, S, a, c) with s_i = a + c d_i (Sec. 3)."""
    d = _c(d, np.float32).ravel()
    S, a, c = _D(), _D(), _D()
    rc = _load().orc_budget_coeffs(_ptr(d), d.size, B, phi, ctypes.byref(S),
                                   ctypes.byref(a), ctypes.byref(c))
    return rc, S.value, a.value, c.value


# --------------------------------------------------------------------------
# a2/a3: stochastic rounding, relaxed ramp, offsets (Sec. 4.2-4.3)
# --------------------------------------------------------------------------
def assign_one(s: float, u: float, lam: float = 10.0, hard: bool = False):
    """(n, w, extra) for one pixel with density s and uniform u."""
    n, w, e = _I64(), _D(), _I()
    _load().orc_assign_one(s, u, lam, int(hard), ctypes.byref(n), ctypes.byref(w), ctypes.byref(e))
    return n.value, w.value, e.value


class Alloc:
    """Result of :func:`alloc` (all arrays flat over the N pixels)."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def alloc(d, B: float, phi: float = 0.125, lam: float = 10.0, hard: bool = False,
          seed: int = 0x5EED, frame: int = 0, u48=None) -> Alloc:
    """Sec. 3 and 4.2-4.3.  u48 (optional, uint64 per pixel) replaces the
    counter-based uniforms by explicit ones, u = u48 2^-48 (the blue-noise
    dither, oracle.bluenoise.uniform48)."""
    d = _c(d, np.float32).ravel()
    N = d.size
    s = np.empty(N, np.float64)
    counts = np.empty(N, np.int64)
    offsets = np.empty(N + 1, np.int64)
    w = np.empty(N, np.float64)
    extra = np.empty(N, np.int32)
    coeffs = np.empty(3, np.float64)
    if u48 is not None:
        u = np.ascontiguousarray(np.asarray(u48, np.uint64).ravel())
        if u.size != N:
            raise ValueError("u48 must have one value per pixel")
        rc = _load().orc_alloc_u48(_ptr(d), N, B, phi, lam, int(hard), _ptr(u), _ptr(s),
                                   _ptr(counts), _ptr(offsets), _ptr(w), _ptr(extra),
                                   _ptr(coeffs))
    else:
        rc = _load().orc_alloc(_ptr(d), N, B, phi, lam, int(hard), seed & 0xFFFFFFFFFFFFFFFF,
                               frame, _ptr(s), _ptr(counts), _ptr(offsets), _ptr(w),
                               _ptr(extra), _ptr(coeffs))
    if rc != OK:
        return Alloc(rc=rc)
    T = int(offsets[N])
    sp = np.empty(T, np.int32)
    _load().orc_sample_list(_ptr(offsets), N, _ptr(sp))
    return Alloc(rc=rc, s=s, counts=counts, offsets=offsets, w=w, extra=extra, T=T,
                 sample_pixel=sp, S=coeffs[0], a=coeffs[1], c=coeffs[2])


# --------------------------------------------------------------------------
# a4: renderer stand-in
# --------------------------------------------------------------------------
def sample_noise(seed: int, frame: int, i: int, k: int) -> float:
    return float(_load().orc_sample_noise(seed & 0xFFFFFFFFFFFFFFFF, frame, i, k))


def render(clean, offsets, seed: int, frame: int) -> np.ndarray:
    """rgb [T][3] for the sample list described by ``offsets``."""
    clean = _c(clean, np.float64)
    offsets = _c(offsets, np.int64)
    N = offsets.size - 1
    assert clean.size == 3 * N
    T = int(offsets[-1])
    rgb = np.empty((T, 3), np.float64)
    _load().orc_render(_ptr(clean), _ptr(offsets), N, seed & 0xFFFFFFFFFFFFFFFF, frame, _ptr(rgb))
    return rgb


# --------------------------------------------------------------------------
# a5: splat + pyramid (Eq. stoch_rnoisy, Eq. app-pyramid)
# --------------------------------------------------------------------------
def splat(offsets, rgb, s, w, extra, W: int, H: int, L: int) -> list[np.ndarray]:
    offsets = _c(offsets, np.int64)
    rgb = _c(rgb, np.float64).reshape(-1, 3)
    s = _c(s, np.float64)
    w = _c(w, np.float64)
    extra = _c(extra, np.int32)
    layers = [np.empty((3, H >> l, W >> l), np.float64) for l in range(L)]
    ptrs = (ctypes.c_void_p * L)(*[a.ctypes.data for a in layers])
    rc = _load().orc_splat(_ptr(offsets), _ptr(rgb), _ptr(s), _ptr(w), _ptr(extra), W, H, L,
                           ctypes.cast(ptrs, ctypes.c_void_p))
    if rc != OK:
        raise ValueError(f"orc_splat rc={rc}")
    return layers


# --------------------------------------------------------------------------
# a6-a8: reconstruction (Appendix A)
# --------------------------------------------------------------------------
def warp(prev, mv) -> np.ndarray:
    """W_t L_{t-1}: prev [3][H][W] (FP64), mv [2][H][W] (FP32 pixels)."""
    prev = _c(prev, np.float64)
    mv = _c(mv, np.float32)
    _, H, W = prev.shape
    out = np.empty_like(prev)
    _load().orc_warp(_ptr(prev), _ptr(mv), W, H, _ptr(out))
    return out


def reconstruct_level(noisy, logits, coarse=None, warped=None, mask=None) -> np.ndarray:
    noisy = _c(noisy, np.float64)
    logits = _c(logits, np.float64)
    _, Hl, Wl = noisy.shape
    C = logits.shape[0]
    coarse = None if coarse is None else _c(coarse, np.float64)
    warped = None if warped is None else _c(warped, np.float64)
    mask = None if mask is None else _c(mask, np.uint8)
    out = np.empty_like(noisy)
    rc = _load().orc_reconstruct_level(_ptr(noisy), _ptr(logits), C, _ptr(coarse), _ptr(warped),
                                       _ptr(mask), Wl, Hl, _ptr(out))
    if rc != OK:
        raise ValueError(f"orc_reconstruct_level rc={rc}")
    return out


def reconstruct(layers, logits, prev=None, mv=None, mask=None):
    """Coarse-to-fine reconstruction: returns (hdr, [L-hat^l for l = 0..L-1])."""
    L = len(layers)
    hats = [None] * L
    for l in range(L - 1, -1, -1):
        coarse = hats[l + 1] if l + 1 < L else None
        warped = None
        m = None
        if l == 0 and prev is not None:
            warped = warp(prev, mv)
            m = mask
        hats[l] = reconstruct_level(layers[l], logits[l], coarse, warped, m)
    return hats[0], hats


# --------------------------------------------------------------------------
# a9: tone map (Sec. 5)
# --------------------------------------------------------------------------
def tau(x: float, s: float = 0.5, h: float = 0.5) -> float:
    return float(_load().orc_tau(x, s, h))


def srgb_encode(v: float) -> float:
    return float(_load().orc_srgb_encode(v))


def tonemap(hdr, alpha=1.0, beta=1.0, k=0.0, s=0.5, h=0.5) -> np.ndarray:
    hdr = _c(hdr, np.float64)
    N = hdr.size // 3
    out = np.empty_like(hdr)
    _load().orc_tonemap(_ptr(hdr), N, alpha, beta, k, s, h, _ptr(out))
    return out


# --------------------------------------------------------------------------
# The whole frame (plain method): alloc -> render -> splat -> reconstruct -> tau
# --------------------------------------------------------------------------
def frame(d, clean, logits, W, H, L, B, *, prev=None, mv=None, mask=None, lam=10.0,
          hard=False, phi=0.125, seed=0x5EED, render_seed=0xC0FFEE, frame_index=0,
          tm=(1.0, 1.0, 0.0, 0.5, 0.5)):
    a = alloc(d, B, phi=phi, lam=lam, hard=hard, seed=seed, frame=frame_index)
    if a.rc != OK:
        raise ValueError(f"alloc rc={a.rc}")
    rgb = render(clean, a.offsets, render_seed, frame_index)
    layers = splat(a.offsets, rgb, a.s, a.w, a.extra, W, H, L)
    hdr, hats = reconstruct(layers, logits, prev=prev, mv=mv, mask=mask)
    ldr = tonemap(hdr, *tm)
    return dict(alloc=a, rgb=rgb, layers=layers, hats=hats, hdr=hdr, ldr=ldr)


# --------------------------------------------------------------------------
# a11: backward (analytic gradients, each pinned by finite differences)
# --------------------------------------------------------------------------
def reconstruct_level_backward(noisy, logits, g, coarse=None, warped=None, mask=None):
    """(grad_logits, grad_noisy, grad_coarse, grad_warped) of loss = sum g * out."""
    noisy = _c(noisy, np.float64)
    logits = _c(logits, np.float64)
    g = _c(g, np.float64)
    _, Hl, Wl = noisy.shape
    C = logits.shape[0]
    coarse = None if coarse is None else _c(coarse, np.float64)
    warped = None if warped is None else _c(warped, np.float64)
    mask = None if mask is None else _c(mask, np.uint8)
    gl = np.empty_like(logits)
    gn = np.zeros_like(noisy)
    gc = None if coarse is None else np.zeros_like(coarse)
    gw = None if warped is None else np.zeros_like(warped)
    rc = _load().orc_reconstruct_level_backward(_ptr(noisy), _ptr(logits), C, _ptr(coarse),
                                                _ptr(warped), _ptr(mask), Wl, Hl, _ptr(g),
                                                _ptr(gl), _ptr(gn), _ptr(gc), _ptr(gw))
    if rc != OK:
        raise ValueError(f"orc_reconstruct_level_backward rc={rc}")
    return gl, gn, gc, gw


def warp_backward(mv, g) -> np.ndarray:
    mv = _c(mv, np.float32)
    g = _c(g, np.float64)
    _, H, W = g.shape
    out = np.zeros_like(g)
    _load().orc_warp_backward(_ptr(mv), W, H, _ptr(g), _ptr(out))
    return out


def tonemap_backward(hdr, grad_ldr, alpha=1.0, beta=1.0, k=0.0, s=0.5, h=0.5) -> np.ndarray:
    hdr = _c(hdr, np.float64)
    grad_ldr = _c(grad_ldr, np.float64)
    out = np.zeros_like(hdr)
    _load().orc_tonemap_backward(_ptr(hdr), hdr.size // 3, alpha, beta, k, s, h, _ptr(grad_ldr),
                                 _ptr(out))
    return out


def l1_loss(ldr, ref):
    """(mean |ldr - ref|, its gradient with respect to ldr)."""
    ldr = _c(ldr, np.float64)
    ref = _c(ref, np.float64)
    grad = np.empty_like(ldr)
    v = _load().orc_l1_loss(_ptr(ldr), _ptr(ref), ldr.size, _ptr(grad))
    return float(v), grad


def pyramid_backward(grad_layers, W, H) -> np.ndarray:
    L = len(grad_layers)
    gls = [_c(a, np.float64) for a in grad_layers]
    out = gls[0].copy()
    ptrs = (ctypes.c_void_p * L)(*[a.ctypes.data for a in gls])
    _load().orc_pyramid_backward(ctypes.cast(ptrs, ctypes.c_void_p), W, H, L, _ptr(out))
    return out


def splat_backward(a: "Alloc", rgb, L0, grad_L0, lam=10.0, hard=False, seed=0x5EED,
                   frame=0) -> np.ndarray:
    rgb = _c(rgb, np.float64).reshape(-1, 3)
    L0 = _c(L0, np.float64)
    grad_L0 = _c(grad_L0, np.float64)
    N = a.s.size
    out = np.empty(N, np.float64)
    _load().orc_splat_backward(_ptr(_c(a.offsets, np.int64)), _ptr(rgb), _ptr(_c(a.s, np.float64)),
                               _ptr(_c(a.extra, np.int32)), N, lam, int(hard),
                               seed & 0xFFFFFFFFFFFFFFFF, frame, _ptr(L0), _ptr(grad_L0), _ptr(out))
    return out


def density_forward(z, B, phi=0.125) -> np.ndarray:
    z = _c(z, np.float64).ravel()
    out = np.empty_like(z)
    _load().orc_density_forward(_ptr(z), z.size, B, phi, _ptr(out))
    return out


def density_backward(z, grad_s, B, phi=0.125) -> np.ndarray:
    z = _c(z, np.float64).ravel()
    grad_s = _c(grad_s, np.float64).ravel()
    out = np.empty_like(z)
    _load().orc_density_backward(_ptr(z), z.size, B, phi, _ptr(grad_s), _ptr(out))
    return out
