"""Thin ctypes binding of the C ABI in ``include/spp.h``.

Argument marshalling only: every function forwards to the entry point of the
same name in ``_build/libspp.so``.  Tensors are passed by device pointer; the
binding checks that they live on a CUDA device, are contiguous and have the
expected dtype, because a host pointer handed to a kernel would fault.  There
is no fallback: importing this module fails loudly when the library has not
been built.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build_lib

if not os.path.exists(build_lib.LIB):
    raise ImportError(
        f"CUDA library {build_lib.LIB} is missing; build it with "
        "`python -c 'import __graft_entry__ as g; g.build()'` (nvcc, sm_103a)")

lib = ctypes.CDLL(build_lib.LIB)

SPP_OK = 0
SPP_ERR_ARG = -1
SPP_ERR_ALIGN = -2
SPP_ERR_SHAPE = -3
SPP_ERR_WORKSPACE = -4
SPP_ERR_CAPACITY = -5
SPP_ERR_TIMEOUT = -6
SPP_ERR_INPUT = -7
SPP_ERR_CUDA = -8

SPP_HOLDOUT_RAMP = 0
SPP_HOLDOUT_HARD = 1
SPP_HOLDOUT_GUMBEL = 2
SPP_HOLDOUT_DASR = 3
SPP_ESTIMATOR_RELAXED = 0
SPP_ESTIMATOR_STRAIGHT_THROUGH = 1
SPP_ESTIMATOR_GUMBEL = 2
SPP_ESTIMATOR_DASR = 3
SPP_FLAG_EXACT_FP64 = 1
SPP_FLAG_TEST_STALL_TILE1 = 1 << 31


class spp_params(ctypes.Structure):
    _fields_ = [("budget", ctypes.c_double), ("uniform_fraction", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("frame", ctypes.c_uint32), ("holdout_mode", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class spp_tonemap(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("beta", ctypes.c_float),
                ("exposure", ctypes.c_float), ("shadow", ctypes.c_float),
                ("highlight", ctypes.c_float)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_U32 = ctypes.c_uint32
_SZ = ctypes.c_size_t

_SIGS = {
    "spp_strerror": (ctypes.c_char_p, [_I]),
    "spp_abi_version": (_I, []),
    "spp_launch_count": (_U64, []),
    "spp_set_dependent_launch": (_I, [_I]),
    "spp_get_dependent_launch": (_I, []),
    "spp_test_stall_reconstruction": (_I, [_I]),
    "spp_get_status": (_I, [_P, _P]),
    "spp_clear_status": (_I, [_P, _P]),
    "spp_alloc_workspace_bytes": (_SZ, [_I, _I]),
    "spp_alloc_sample_map": (_I, [_P, _I, _I, ctypes.POINTER(spp_params), _P, _P, _P, _I64, _P,
                                  _P, _P, _P, _P, _SZ, _P]),
    "spp_alloc_sample_map_static": (_I, [_P, _I, _I, ctypes.POINTER(spp_params), _P, _P, _P,
                                         _I64, _P, _P, _P, _P, _P]),
    "spp_render_synthetic": (_I, [_P, _P, _P, _P, _I64, _I, _I, _U64, _U32, _P, _P]),
    "spp_splat_samples": (_I, [_P, _P, _P, _P, _I64, _I, _I, _I, _P, _P]),
    "spp_reconstruct_workspace_bytes": (_SZ, [_I, _I, _I]),
    "spp_warp_previous": (_I, [_P, _P, _I, _I, _P, _P]),
    "spp_reconstruct_level": (_I, [_P, _P, _I, _P, _P, _P, _I, _I,
                                   ctypes.POINTER(spp_tonemap), _P, _P, _P, _P]),
    "spp_reconstruct_frame": (_I, [_P, _P, _I, _P, _P, _P, _I, _I, _I,
                                   ctypes.POINTER(spp_tonemap), _P, _P, _P, _SZ, _P, _P]),
    "spp_reconstruct_level_backward": (_I, [_P, _P, _I, _P, _P, _P, _I, _I, _P, _P, _P, _P, _P,
                                            _P]),
    "spp_warp_previous_backward": (_I, [_P, _I, _I, _P, _P, _P]),
    "spp_tonemap_backward": (_I, [_P, _I, _I, ctypes.POINTER(spp_tonemap), _P, _P, _P]),
    "spp_l1_loss": (_I, [_P, _P, _I64, _P, _P, _P]),
    "spp_pyramid_backward": (_I, [_P, _I, _I, _I, _P, _P]),
    "spp_splat_backward": (_I, [_P, _P, _P, _P, _P, _P, _I64, _I, _I, ctypes.POINTER(spp_params),
                                _P, _P]),
    "spp_density_backward_workspace_bytes": (_SZ, []),
    "spp_density_backward": (_I, [_P, _I64, ctypes.c_double, ctypes.c_double, _P, _P, _P, _SZ,
                                  _P]),
    "spp_unet_layer": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "spp_unet_param_count": (_I64, []),
    "spp_unet_packed_bytes": (_SZ, [_I]),
    "spp_unet_pack": (_I, [_P, _I, _P, _SZ, _P]),
    "spp_assemble_features": (_I, [_P, _P, _P, _P, _P, _I, _I, _P, _P]),
    "spp_predict_workspace_bytes": (_SZ, [_I, _I, _I]),
    "spp_predict_density_and_kernels": (_I, [_P, _P, _I, _I, _I, _P, _P, _P, _P, _P, _SZ, _P,
                                             _P]),
    "spp_conv3x3_workspace_bytes": (_SZ, [_I, _I]),
    "spp_conv3x3_forward": (_I, [_P, _I, _I, _I, _I, _I, _P, _P, _I, _P, _P, _SZ, _P, _P]),
    "spp_conv3x3_backward_data": (_I, [_P, _I, _I, _I, _I, _I, _P, _P, _P, _P, _SZ, _P, _P]),
    "spp_conv3x3_backward_weights_workspace_bytes": (_SZ, [_I, _I, _I, _I, _I]),
    "spp_conv3x3_backward_weights": (_I, [_P, _P, _I, _I, _I, _I, _I, _P, _P, _P, _SZ, _P, _P]),
    "spp_unet_backward_workspace_bytes": (_SZ, [_I, _I, _I]),
    "spp_unet_backward": (_I, [_P, _P, _I, _I, _I, _P, _SZ, _P, _P, _P, _P, _P, _SZ, _P, _P]),
    "spp_adamw_step": (_I, [_P, _P, _P, _P, _I64, _I, ctypes.c_float, ctypes.c_float,
                            ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P]),
    "spp_tonemap_image": (_I, [_P, _I, _I, ctypes.POINTER(spp_tonemap), _P, _P]),
    "spp_mse": (_I, [_P, _P, _I64, _P, _P]),
    "spp_blue_noise_mask": (_I, [_I, _U64, _P]),
    "spp_alloc_sample_map_dithered": (_I, [_P, _I, _I, ctypes.POINTER(spp_params), _P, _I, _P,
                                           _P, _P, _I64, _P, _P, _P, _P, _P, _SZ, _P]),
    "spp_combined_loss": (_I, [_P, _P, _P, _P, _I64, ctypes.c_float, ctypes.c_float, _P, _P,
                               _P]),
    "spp_net_spec": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                          ctypes.POINTER(_I)]),
    "spp_net_layer": (_I, [_I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "spp_net_param_count": (_I64, [_I]),
    "spp_net_packed_bytes": (_SZ, [_I, _I]),
    "spp_net_pack": (_I, [_I, _P, _I, _P, _SZ, _P]),
    "spp_net_workspace_bytes": (_SZ, [_I, _I, _I, _I]),
    "spp_net_forward": (_I, [_I, _P, _P, _I, _I, _I, _P, _P, _P, _P, _SZ, _P, _P]),
    "spp_net_backward_workspace_bytes": (_SZ, [_I, _I, _I, _I]),
    "spp_net_backward": (_I, [_I, _P, _I, _I, _I, _P, _SZ, _P, _P, _P, _P, _P, _P, _SZ, _P,
                              _P]),
    "spp_density_softmax_workspace_bytes": (_SZ, [_I]),
    "spp_density_softmax": (_I, [_P, _I, _I, _I, _I64, _P, _P, _SZ, _P]),
    "spp_warp_latent": (_I, [_P, _P, _I, _I, _P, _P]),
    "spp_assemble_sampler_features": (_I, [_P, _P, _P, _P, _P, _P, _I, _I, _P, _P]),
    "spp_assemble_denoiser_features": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _I, _P,
                                            _P]),
    "spp_denoiser_features_backward": (_I, [_P, _P, _P, _I, _I, _P, _P, _P]),
    "spp_demodulate": (_I, [_P, _P, _P, _I, _I, _I, _P, _P, _P, _P]),
    "spp_remodulate_tonemap": (_I, [_P, _P, _I, _I, ctypes.POINTER(spp_tonemap), _P, _P, _P]),
    "spp_remodulate_backward": (_I, [_P, _P, _I, _I, _P, _P]),
    "spp_demodulate_backward": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _I, _I, _P, _P, _P]),
    "spp_alloc_sample_map_systematic": (_I, [_P, _I, _I, ctypes.POINTER(spp_params), _P, _P, _P,
                                             _I64, _P, _P, _P, _P, _P, _SZ, _P]),
    "spp_density_lowres": (_I, [_P, _I, _I, _I, _P, _P]),
    "spp_latent_tanh": (_I, [_P, _I, _I, _P, _P]),
    "spp_net_input_layout": (_I, [_I, _I, _I, _I, ctypes.POINTER(_SZ), ctypes.POINTER(_I)]),
    "spp_net_forward_prepared": (_I, [_I, _P, _I, _I, _I, _P, _P, _P, _P, _SZ, _P, _P]),
    "spp_assemble_sampler_input": (_I, [_P, _P, _P, _P, _P, _P, _I, _I, _P, _P]),
    "spp_assemble_denoiser_input": (_I, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _I, _P, _P]),
    "spp_warp_channels": (_I, [_P, _I, _P, _I, _I, _P, _P]),
    "spp_splat_backward_estimator": (_I, [_P, _P, _P, _P, _P, _P, _P, _I64, _I, _I,
                                          ctypes.POINTER(spp_params), _I, _P, _U64, _P, _P]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class SppError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        super().__init__(f"{where}: {spp_strerror(code)} ({code})")


def check(code: int, where: str = "spp") -> int:
    if code != SPP_OK:
        raise SppError(code, where)
    return code


def _dev(t: torch.Tensor | None, dtype: torch.dtype | None = None):
    """Device pointer of a contiguous CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr_array(ts, dtype):
    arr = (ctypes.c_void_p * len(ts))(*[_dev(t, dtype).value for t in ts])
    return arr


def spp_strerror(code: int) -> str:
    return lib.spp_strerror(code).decode()


def spp_abi_version() -> int:
    return lib.spp_abi_version()


def spp_launch_count() -> int:
    return int(lib.spp_launch_count())


def spp_set_dependent_launch(on: bool) -> bool:
    """Turns programmatic dependent launch on or off; returns the previous setting."""
    return bool(lib.spp_set_dependent_launch(1 if on else 0))


def spp_get_dependent_launch() -> bool:
    return bool(lib.spp_get_dependent_launch())


def spp_test_stall_reconstruction(tile: int) -> int:
    """Test of the bounded waits: the next pipelined reconstruction launch
    issues no copies for tile `tile` (-1 cancels)."""
    return lib.spp_test_stall_reconstruction(tile)


def spp_get_status(status: torch.Tensor, stream=None) -> int:
    return lib.spp_get_status(_dev(status, torch.int32), _stream(stream))


def spp_clear_status(status: torch.Tensor, stream=None) -> int:
    return lib.spp_clear_status(_dev(status, torch.int32), _stream(stream))


def spp_alloc_workspace_bytes(W: int, H: int) -> int:
    return int(lib.spp_alloc_workspace_bytes(W, H))


def make_params(budget: float, *, uniform_fraction: float = 0.125, lam: float = 10.0,
                seed: int = 0x5EED, frame: int = 0, hard: bool = False, gumbel: bool = False,
                dasr: bool = False, exact_fp64: bool = False) -> spp_params:
    mode = (SPP_HOLDOUT_DASR if dasr else SPP_HOLDOUT_GUMBEL if gumbel
            else SPP_HOLDOUT_HARD if hard else SPP_HOLDOUT_RAMP)
    return spp_params(budget, uniform_fraction, lam, seed & 0xFFFFFFFFFFFFFFFF, frame, mode,
                      SPP_FLAG_EXACT_FP64 if exact_fp64 else 0, 0)


def make_tonemap(alpha=1.0, beta=1.0, exposure=0.0, shadow=0.5, highlight=0.5) -> spp_tonemap:
    return spp_tonemap(alpha, beta, exposure, shadow, highlight)


def spp_alloc_sample_map(d, W, H, params: spp_params, counts, offsets, sample_pixel, capacity,
                         s_out, holdout_w, total, status, ws, stream=None) -> int:
    return lib.spp_alloc_sample_map(
        _dev(d, torch.float32), W, H, ctypes.byref(params), _dev(counts, torch.int32),
        _dev(offsets, torch.int32), _dev(sample_pixel, torch.int32), int(capacity),
        _dev(s_out, torch.float32), _dev(holdout_w, torch.float32), _dev(total, torch.int64),
        _dev(status, torch.int32), _dev(ws), ws.numel() * ws.element_size(), _stream(stream))


def spp_alloc_sample_map_static(d, W, H, params: spp_params, counts, offsets, sample_pixel,
                                capacity, s_out, holdout_w, total, status, stream=None) -> int:
    return lib.spp_alloc_sample_map_static(
        _dev(d, torch.float32), W, H, ctypes.byref(params), _dev(counts, torch.int32),
        _dev(offsets, torch.int32), _dev(sample_pixel, torch.int32), int(capacity),
        _dev(s_out, torch.float32), _dev(holdout_w, torch.float32), _dev(total, torch.int64),
        _dev(status, torch.int32), _stream(stream))


def spp_render_synthetic(clean, offsets, sample_pixel, total, capacity, W, H, seed, frame, rgb,
                         stream=None) -> int:
    return lib.spp_render_synthetic(
        _dev(clean, torch.float32), _dev(offsets, torch.int32), _dev(sample_pixel, torch.int32),
        _dev(total, torch.int64), int(capacity), W, H, seed & 0xFFFFFFFFFFFFFFFF, frame,
        _dev(rgb, torch.float32), _stream(stream))


def spp_splat_samples(offsets, rgb, s, holdout_w, capacity, W, H, L, layers, stream=None) -> int:
    arr = _ptr_array(layers, torch.float32)
    return lib.spp_splat_samples(
        _dev(offsets, torch.int32), _dev(rgb, torch.float32), _dev(s, torch.float32),
        _dev(holdout_w, torch.float32), int(capacity), W, H, L, ctypes.cast(arr, _P),
        _stream(stream))


def spp_reconstruct_workspace_bytes(W: int, H: int, L: int) -> int:
    return int(lib.spp_reconstruct_workspace_bytes(W, H, L))


def spp_warp_previous(prev_hdr, mv, W, H, warped, stream=None) -> int:
    return lib.spp_warp_previous(_dev(prev_hdr, torch.float32), _dev(mv, torch.float32), W, H,
                                 _dev(warped, torch.float32), _stream(stream))


def spp_reconstruct_level(noisy, logits, C, coarse, warped_prev, mask, Wl, Hl, tm, out, out_ldr,
                          status=None, stream=None) -> int:
    return lib.spp_reconstruct_level(
        _dev(noisy, torch.float32), _dev(logits, torch.float32), C, _dev(coarse, torch.float32),
        _dev(warped_prev, torch.float32), _dev(mask, torch.uint8), Wl, Hl,
        ctypes.byref(tm) if tm is not None else None, _dev(out, torch.float32),
        _dev(out_ldr, torch.float32), _dev(status, torch.int32), _stream(stream))


def spp_reconstruct_frame(layers, logits, C0, prev_hdr, mv, mask, W, H, L, tm, out_hdr, out_ldr,
                          ws, status=None, stream=None) -> int:
    la = _ptr_array(layers, torch.float32)
    lo = _ptr_array(logits, torch.float32)
    return lib.spp_reconstruct_frame(
        ctypes.cast(la, _P), ctypes.cast(lo, _P), C0, _dev(prev_hdr, torch.float32),
        _dev(mv, torch.float32), _dev(mask, torch.uint8), W, H, L,
        ctypes.byref(tm) if tm is not None else None, _dev(out_hdr, torch.float32),
        _dev(out_ldr, torch.float32), _dev(ws) if ws is not None else None,
        (ws.numel() * ws.element_size()) if ws is not None else 0, _dev(status, torch.int32),
        _stream(stream))


# --------------------------------------------------------------------------
# backward entry points
# --------------------------------------------------------------------------
def spp_reconstruct_level_backward(noisy, logits, C, coarse, warped_prev, mask, Wl, Hl, grad_out,
                                   grad_logits, grad_noisy, grad_coarse, grad_warped,
                                   stream=None) -> int:
    f = torch.float32
    return lib.spp_reconstruct_level_backward(
        _dev(noisy, f), _dev(logits, f), C, _dev(coarse, f), _dev(warped_prev, f),
        _dev(mask, torch.uint8), Wl, Hl, _dev(grad_out, f), _dev(grad_logits, f),
        _dev(grad_noisy, f), _dev(grad_coarse, f), _dev(grad_warped, f), _stream(stream))


def spp_warp_previous_backward(mv, W, H, grad_warped, grad_prev, stream=None) -> int:
    f = torch.float32
    return lib.spp_warp_previous_backward(_dev(mv, f), W, H, _dev(grad_warped, f),
                                          _dev(grad_prev, f), _stream(stream))


def spp_tonemap_backward(hdr, W, H, tm, grad_ldr, grad_hdr, stream=None) -> int:
    f = torch.float32
    return lib.spp_tonemap_backward(_dev(hdr, f), W, H,
                                    ctypes.byref(tm) if tm is not None else None,
                                    _dev(grad_ldr, f), _dev(grad_hdr, f), _stream(stream))


def spp_l1_loss(ldr, ref, n, loss, grad_ldr, stream=None) -> int:
    f = torch.float32
    return lib.spp_l1_loss(_dev(ldr, f), _dev(ref, f), int(n), _dev(loss, f), _dev(grad_ldr, f),
                           _stream(stream))


def spp_pyramid_backward(grad_layers, W, H, L, grad_L0, stream=None) -> int:
    arr = (ctypes.c_void_p * L)(*[0 if l == 0 else _dev(grad_layers[l], torch.float32).value
                                   for l in range(L)])
    return lib.spp_pyramid_backward(ctypes.cast(arr, _P), W, H, L, _dev(grad_L0, torch.float32),
                                    _stream(stream))


def spp_splat_backward(offsets, counts, rgb, s, layer0, grad_layer0, capacity, W, H,
                       params: spp_params, grad_s, stream=None) -> int:
    f = torch.float32
    return lib.spp_splat_backward(
        _dev(offsets, torch.int32), _dev(counts, torch.int32), _dev(rgb, f), _dev(s, f),
        _dev(layer0, f), _dev(grad_layer0, f), int(capacity), W, H, ctypes.byref(params),
        _dev(grad_s, f), _stream(stream))


def spp_density_backward_workspace_bytes() -> int:
    return int(lib.spp_density_backward_workspace_bytes())


def spp_density_backward(d, N, budget, uniform_fraction, grad_s, grad_z, ws, stream=None) -> int:
    f = torch.float32
    return lib.spp_density_backward(_dev(d, f), int(N), float(budget), float(uniform_fraction),
                                    _dev(grad_s, f), _dev(grad_z, f), _dev(ws),
                                    ws.numel() * ws.element_size(), _stream(stream))


# ------------------------------------------------------------ a10: predictor
def _nbytes(t):
    return t.numel() * t.element_size()


def spp_unet_layer(i: int):
    """(cin, cout, relu) of layer i."""
    a, b, c = _I(), _I(), _I()
    check(lib.spp_unet_layer(i, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "layer")
    return a.value, b.value, c.value


def spp_unet_param_count() -> int:
    return int(lib.spp_unet_param_count())


def spp_unet_packed_bytes(with_backward: bool) -> int:
    return int(lib.spp_unet_packed_bytes(int(with_backward)))


def spp_unet_pack(theta, with_backward, packed, stream=None) -> int:
    return lib.spp_unet_pack(_dev(theta, torch.float32), int(with_backward), _dev(packed),
                             _nbytes(packed), _stream(stream))


def spp_assemble_features(albedo, normal, depth, mv, prev_ldr, W, H, in12, stream=None) -> int:
    f = torch.float32
    return lib.spp_assemble_features(_dev(albedo, f), _dev(normal, f), _dev(depth, f), _dev(mv, f),
                                     _dev(prev_ldr, f), W, H, _dev(in12, f), _stream(stream))


def spp_predict_workspace_bytes(B: int, W: int, H: int) -> int:
    return int(lib.spp_predict_workspace_bytes(B, W, H))


def spp_predict_density_and_kernels(packed, in12, B, W, H, density, logits0, logits1, logits2,
                                    ws, status, stream=None) -> int:
    f = torch.float32
    return lib.spp_predict_density_and_kernels(
        _dev(packed), _dev(in12, f), B, W, H, _dev(density, f), _dev(logits0, f),
        _dev(logits1, f), _dev(logits2, f), _dev(ws), _nbytes(ws), _dev(status, torch.int32),
        _stream(stream))


def spp_conv3x3_workspace_bytes(cin: int, cout: int) -> int:
    return int(lib.spp_conv3x3_workspace_bytes(cin, cout))


def spp_conv3x3_forward(x, B, W, H, cin, cout, w, bias, relu, y, ws, status, stream=None) -> int:
    bf = torch.bfloat16
    return lib.spp_conv3x3_forward(_dev(x, bf), B, W, H, cin, cout, _dev(w, torch.float32),
                                   _dev(bias, torch.float32), int(relu), _dev(y, bf), _dev(ws),
                                   _nbytes(ws), _dev(status, torch.int32), _stream(stream))


def spp_conv3x3_backward_data(g, B, W, H, cin, cout, w, act, gx, ws, status, stream=None) -> int:
    bf = torch.bfloat16
    return lib.spp_conv3x3_backward_data(_dev(g, bf), B, W, H, cin, cout, _dev(w, torch.float32),
                                         _dev(act, bf), _dev(gx, bf), _dev(ws), _nbytes(ws),
                                         _dev(status, torch.int32), _stream(stream))


def spp_conv3x3_backward_weights_workspace_bytes(B, W, H, cin, cout) -> int:
    return int(lib.spp_conv3x3_backward_weights_workspace_bytes(B, W, H, cin, cout))


def spp_conv3x3_backward_weights(x, g, B, W, H, cin, cout, gw, gb, ws, status, stream=None) -> int:
    bf, f = torch.bfloat16, torch.float32
    return lib.spp_conv3x3_backward_weights(_dev(x, bf), _dev(g, bf), B, W, H, cin, cout,
                                            _dev(gw, f), _dev(gb, f), _dev(ws), _nbytes(ws),
                                            _dev(status, torch.int32), _stream(stream))


# ------------------------------------------------------------ a11: training
def spp_unet_backward_workspace_bytes(B: int, W: int, H: int) -> int:
    return int(lib.spp_unet_backward_workspace_bytes(B, W, H))


def spp_unet_backward(packed, in12, B, W, H, fwd_ws, g0, g1, g2, grad_theta, ws, status,
                      stream=None) -> int:
    f = torch.float32
    return lib.spp_unet_backward(_dev(packed), _dev(in12, f), B, W, H, _dev(fwd_ws),
                                 _nbytes(fwd_ws), _dev(g0, f), _dev(g1, f), _dev(g2, f),
                                 _dev(grad_theta, f), _dev(ws), _nbytes(ws),
                                 _dev(status, torch.int32), _stream(stream))


def spp_adamw_step(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                   weight_decay=1e-4, grad_scale=1.0, stream=None) -> int:
    f = torch.float32
    return lib.spp_adamw_step(_dev(theta, f), _dev(grad, f), _dev(m, f), _dev(v, f),
                              theta.numel(), int(step), lr, beta1, beta2, eps, weight_decay,
                              grad_scale, _stream(stream))


def spp_tonemap_image(hdr, W, H, tm, ldr, stream=None) -> int:
    f = torch.float32
    return lib.spp_tonemap_image(_dev(hdr, f), W, H, ctypes.byref(tm), _dev(ldr, f),
                                 _stream(stream))


def spp_mse(a, b, n, out, stream=None) -> int:
    f = torch.float32
    return lib.spp_mse(_dev(a, f), _dev(b, f), int(n), _dev(out, torch.float64), _stream(stream))


def spp_combined_loss(ldr, ref, prev_warped, ref_prev_warped, n, temporal_weight, spatial_weight,
                      loss, grad_ldr, stream=None) -> int:
    f = torch.float32
    return lib.spp_combined_loss(_dev(ldr, f), _dev(ref, f), _dev(prev_warped, f),
                                 _dev(ref_prev_warped, f), int(n), float(temporal_weight),
                                 float(spatial_weight), _dev(loss, f), _dev(grad_ldr, f),
                                 _stream(stream))


# ------------------------------------------------------ blue-noise dithering
def spp_blue_noise_mask(T: int, seed: int):
    """The T x T rank matrix as a host numpy uint16 array."""
    import numpy as np
    out = np.empty((T, T), np.uint16)
    check(lib.spp_blue_noise_mask(T, seed & 0xFFFFFFFFFFFFFFFF,
                                  ctypes.c_void_p(out.ctypes.data)), "spp_blue_noise_mask")
    return out


def spp_alloc_sample_map_dithered(d, W, H, params: spp_params, mask, counts, offsets,
                                  sample_pixel, capacity, s_out, holdout_w, total, status, ws,
                                  stream=None) -> int:
    return lib.spp_alloc_sample_map_dithered(
        _dev(d, torch.float32), W, H, ctypes.byref(params), _dev(mask, torch.int16),
        mask.shape[0], _dev(counts, torch.int32), _dev(offsets, torch.int32),
        _dev(sample_pixel, torch.int32), int(capacity), _dev(s_out, torch.float32),
        _dev(holdout_w, torch.float32), _dev(total, torch.int64), _dev(status, torch.int32),
        _dev(ws), _nbytes(ws), _stream(stream))


# ------------------------------------------- f1: two-stage pipeline
SPP_NET_JOINT = 0
SPP_NET_SAMPLER = 1
SPP_NET_DENOISER = 2
SPP_LATENT_CHANNELS = 7
SPP_DEMOD_PLANE = 54
SPP_LATENT_PLANE = 57


def spp_net_spec(net: int):
    """(cin, (h0, h1, h2)) of network `net`."""
    a, b, c, d = _I(), _I(), _I(), _I()
    check(lib.spp_net_spec(net, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                           ctypes.byref(d)), "spp_net_spec")
    return a.value, (b.value, c.value, d.value)


def spp_net_layer(net: int, i: int):
    a, b, c = _I(), _I(), _I()
    check(lib.spp_net_layer(net, i, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
          "spp_net_layer")
    return a.value, b.value, c.value


def spp_net_param_count(net: int) -> int:
    return int(lib.spp_net_param_count(net))


def spp_net_packed_bytes(net: int, with_backward: bool) -> int:
    return int(lib.spp_net_packed_bytes(net, int(with_backward)))


def spp_net_pack(net, theta, with_backward, packed, stream=None) -> int:
    return lib.spp_net_pack(net, _dev(theta, torch.float32), int(with_backward), _dev(packed),
                            _nbytes(packed), _stream(stream))


def spp_net_workspace_bytes(net: int, B: int, W: int, H: int) -> int:
    return int(lib.spp_net_workspace_bytes(net, B, W, H))


def spp_net_forward(net, packed, x, B, W, H, head0, head1, head2, ws, status, stream=None) -> int:
    f = torch.float32
    return lib.spp_net_forward(net, _dev(packed), _dev(x, f), B, W, H, _dev(head0, f),
                               _dev(head1, f), _dev(head2, f), _dev(ws), _nbytes(ws),
                               _dev(status, torch.int32), _stream(stream))


def spp_net_backward_workspace_bytes(net: int, B: int, W: int, H: int) -> int:
    return int(lib.spp_net_backward_workspace_bytes(net, B, W, H))


def spp_net_backward(net, packed, B, W, H, fwd_ws, g0, g1, g2, grad_theta, grad_in, ws, status,
                     stream=None) -> int:
    f = torch.float32
    return lib.spp_net_backward(net, _dev(packed), B, W, H, _dev(fwd_ws), _nbytes(fwd_ws),
                                _dev(g0, f), _dev(g1, f), _dev(g2, f), _dev(grad_theta, f),
                                _dev(grad_in, f), _dev(ws), _nbytes(ws), _dev(status, torch.int32),
                                _stream(stream))


def spp_density_softmax_workspace_bytes(B: int) -> int:
    return int(lib.spp_density_softmax_workspace_bytes(B))


def spp_density_softmax(z, B, W, H, batch_stride, density, ws, stream=None) -> int:
    f = torch.float32
    return lib.spp_density_softmax(_dev(z, f), B, W, H, int(batch_stride), _dev(density, f),
                                   _dev(ws), _nbytes(ws), _stream(stream))


def spp_warp_latent(raw, mv, W, H, out, stream=None) -> int:
    f = torch.float32
    return lib.spp_warp_latent(_dev(raw, f), _dev(mv, f), W, H, _dev(out, f), _stream(stream))


def spp_assemble_sampler_features(albedo, normal, depth, mv, warped_prev_ldr, warped_latent, W, H,
                                  in19, stream=None) -> int:
    f = torch.float32
    return lib.spp_assemble_sampler_features(_dev(albedo, f), _dev(normal, f), _dev(depth, f),
                                             _dev(mv, f), _dev(warped_prev_ldr, f),
                                             _dev(warped_latent, f), W, H, _dev(in19, f),
                                             _stream(stream))


def spp_assemble_denoiser_features(L0, s, counts, albedo, normal, depth, mv, warped_prev_hdr,
                                   warped_latent, W, H, in24, stream=None) -> int:
    f = torch.float32
    return lib.spp_assemble_denoiser_features(
        _dev(L0, f), _dev(s, f), _dev(counts, torch.int32), _dev(albedo, f), _dev(normal, f),
        _dev(depth, f), _dev(mv, f), _dev(warped_prev_hdr, f), _dev(warped_latent, f), W, H,
        _dev(in24, f), _stream(stream))


def spp_denoiser_features_backward(L0, s, grad_in24, W, H, grad_L0, grad_s, stream=None) -> int:
    f = torch.float32
    return lib.spp_denoiser_features_backward(_dev(L0, f), _dev(s, f), _dev(grad_in24, f), W, H,
                                              _dev(grad_L0, f), _dev(grad_s, f), _stream(stream))


def spp_demodulate(L0, c, warped, W, H, L, m, layers, warped_out, stream=None) -> int:
    f = torch.float32
    arr = _ptr_array(layers[:L], f)
    return lib.spp_demodulate(_dev(L0, f), _dev(c, f), _dev(warped, f), W, H, L, _dev(m, f),
                              ctypes.cast(arr, _P), _dev(warped_out, f), _stream(stream))


def spp_remodulate_tonemap(R, m, W, H, tm, out_hdr, out_ldr, stream=None) -> int:
    f = torch.float32
    return lib.spp_remodulate_tonemap(_dev(R, f), _dev(m, f), W, H, ctypes.byref(tm),
                                      _dev(out_hdr, f), _dev(out_ldr, f), _stream(stream))


def spp_remodulate_backward(grad_out, m, W, H, grad_R, stream=None) -> int:
    f = torch.float32
    return lib.spp_remodulate_backward(_dev(grad_out, f), _dev(m, f), W, H, _dev(grad_R, f),
                                       _stream(stream))


def spp_demodulate_backward(out_hdr, grad_out, L0d, grad_L0d, Wd, grad_Wd, c, m, W, H, grad_L0,
                            grad_c, stream=None) -> int:
    f = torch.float32
    return lib.spp_demodulate_backward(_dev(out_hdr, f), _dev(grad_out, f), _dev(L0d, f),
                                       _dev(grad_L0d, f), _dev(Wd, f), _dev(grad_Wd, f),
                                       _dev(c, f), _dev(m, f), W, H, _dev(grad_L0, f),
                                       _dev(grad_c, f), _stream(stream))


# ------------------------------------------------- f4: pipeline variants
def spp_alloc_sample_map_systematic(d, W, H, params: spp_params, counts, offsets, sample_pixel,
                                    capacity, s_out, holdout_w, total, status, ws,
                                    stream=None) -> int:
    return lib.spp_alloc_sample_map_systematic(
        _dev(d, torch.float32), W, H, ctypes.byref(params), _dev(counts, torch.int32),
        _dev(offsets, torch.int32), _dev(sample_pixel, torch.int32), int(capacity),
        _dev(s_out, torch.float32), _dev(holdout_w, torch.float32), _dev(total, torch.int64),
        _dev(status, torch.int32), _dev(ws), _nbytes(ws), _stream(stream))


def spp_density_lowres(d, W, H, factor, out, stream=None) -> int:
    f = torch.float32
    return lib.spp_density_lowres(_dev(d, f), W, H, int(factor), _dev(out, f), _stream(stream))


def spp_splat_backward_estimator(offsets, counts, rgb, s, layer0, grad_layer0, holdout_w, capacity,
                                 W, H, params: spp_params, estimator: int, clean, render_seed,
                                 grad_s, stream=None) -> int:
    f = torch.float32
    return lib.spp_splat_backward_estimator(
        _dev(offsets, torch.int32), _dev(counts, torch.int32), _dev(rgb, f), _dev(s, f),
        _dev(layer0, f), _dev(grad_layer0, f), _dev(holdout_w, f), int(capacity), W, H,
        ctypes.byref(params), int(estimator), _dev(clean, f), render_seed & 0xFFFFFFFFFFFFFFFF,
        _dev(grad_s, f), _stream(stream))


def spp_latent_tanh(raw, W, H, out, stream=None) -> int:
    f = torch.float32
    return lib.spp_latent_tanh(_dev(raw, f), W, H, _dev(out, f), _stream(stream))


def spp_warp_channels(src, C, mv, W, H, out, stream=None) -> int:
    f = torch.float32
    return lib.spp_warp_channels(_dev(src, f), int(C), _dev(mv, f), W, H, _dev(out, f),
                                 _stream(stream))


def spp_net_input_layout(net: int, B_: int, W: int, H: int):
    """(byte offset, channels) of the BF16 NHWC input copy in the forward workspace."""
    off, ch = _SZ(), _I()
    check(lib.spp_net_input_layout(net, B_, W, H, ctypes.byref(off), ctypes.byref(ch)),
          "spp_net_input_layout")
    return off.value, ch.value


def spp_net_forward_prepared(net, packed, B_, W, H, head0, head1, head2, ws, status,
                             stream=None) -> int:
    f = torch.float32
    return lib.spp_net_forward_prepared(net, _dev(packed), B_, W, H, _dev(head0, f),
                                        _dev(head1, f), _dev(head2, f), _dev(ws), _nbytes(ws),
                                        _dev(status, torch.int32), _stream(stream))


def spp_assemble_sampler_input(albedo, normal, depth, mv, warped_prev_ldr, warped_latent, W, H,
                               x_nhwc32, stream=None) -> int:
    f = torch.float32
    return lib.spp_assemble_sampler_input(_dev(albedo, f), _dev(normal, f), _dev(depth, f),
                                          _dev(mv, f), _dev(warped_prev_ldr, f),
                                          _dev(warped_latent, f), W, H,
                                          _dev(x_nhwc32, torch.bfloat16), _stream(stream))


def spp_assemble_denoiser_input(L0, s, counts, albedo, normal, depth, mv, warped_prev_hdr,
                                warped_latent, W, H, x_nhwc32, stream=None) -> int:
    f = torch.float32
    return lib.spp_assemble_denoiser_input(
        _dev(L0, f), _dev(s, f), _dev(counts, torch.int32), _dev(albedo, f), _dev(normal, f),
        _dev(depth, f), _dev(mv, f), _dev(warped_prev_hdr, f), _dev(warped_latent, f), W, H,
        _dev(x_nhwc32, torch.bfloat16), _stream(stream))
