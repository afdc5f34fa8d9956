"""The C-ABI library loads and exports every entry point of include/spp.h.

CPU only: nothing here launches a kernel.  The argument checks below return
before any CUDA call, so they run without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spp.h")


@pytest.fixture(scope="module")
def lib():
    from conftest import build_spp_lib
    return ctypes.CDLL(build_spp_lib())


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    syms = declared_symbols()
    for name in ("spp_alloc_sample_map", "spp_render_synthetic", "spp_splat_samples",
                 "spp_reconstruct_frame", "spp_reconstruct_level", "spp_get_status"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_status_strings_and_version():
    import paper_2602_08642_gb300 as spp
    assert spp.spp_abi_version() == 7
    for code in range(0, -9, -1):
        assert spp.spp_strerror(code) and spp.spp_strerror(code) != "unknown status code"
    assert spp.spp_strerror(-99) == "unknown status code"


def test_dependent_launch_switch():
    import paper_2602_08642_gb300._binding as B
    assert B.spp_get_dependent_launch()  # on by default
    assert B.spp_set_dependent_launch(False) is True
    assert B.spp_get_dependent_launch() is False
    assert B.spp_set_dependent_launch(True) is False
    assert B.spp_get_dependent_launch()


def test_workspace_queries():
    import paper_2602_08642_gb300 as spp
    assert spp.spp_alloc_workspace_bytes(1920, 1080) == 256 + 8 * ((1920 * 1080 + 2047) // 2048)
    assert spp.spp_alloc_workspace_bytes(-1, 4) == 0
    b = spp.spp_reconstruct_workspace_bytes(1920, 1080, 3)
    assert b >= 3 * 4 * (1920 * 1080 + 960 * 540 + 480 * 270)
    assert spp.spp_reconstruct_workspace_bytes(64, 64, 1) == 0
    assert spp.spp_reconstruct_workspace_bytes(64, 64, 6) == 0


def _fake(addr):
    return ctypes.c_void_p(addr)


def test_host_argument_errors(lib):
    """Host-side validation returns before any CUDA call."""
    import paper_2602_08642_gb300._binding as B
    p = B.make_params(0.25)
    a = _fake(0x10000)
    mis = _fake(0x10004)
    n = None
    f = B.lib.spp_alloc_sample_map
    # null params / negative size
    assert f(a, 4, 4, None, a, a, a, 16, a, a, a, a, a, 4096, n) == B.SPP_ERR_ARG
    assert f(a, -1, 4, ctypes.byref(p), a, a, a, 16, a, a, a, a, a, 4096, n) == B.SPP_ERR_ARG
    # misaligned density
    assert f(mis, 4, 4, ctypes.byref(p), a, a, a, 16, a, a, a, a, a, 4096, n) == B.SPP_ERR_ALIGN
    # workspace too small
    assert f(a, 64, 64, ctypes.byref(p), a, a, a, 16, a, a, a, a, a, 8, n) == B.SPP_ERR_WORKSPACE
    # bad budget, lambda, mode, reserved
    for bad in (B.make_params(0.0), B.make_params(-1.0), B.make_params(0.25, lam=0.5)):
        assert f(a, 4, 4, ctypes.byref(bad), a, a, a, 16, a, a, a, a, a, 4096, n) == B.SPP_ERR_ARG
    q = B.make_params(0.25)
    q.reserved = 1
    assert f(a, 4, 4, ctypes.byref(q), a, a, a, 16, a, a, a, a, a, 4096, n) == B.SPP_ERR_ARG
    # budget * N beyond int32 sample indices
    big = B.make_params(2000.0)
    assert f(a, 4096, 4096, ctypes.byref(big), a, a, a, 16, a, a, a, a, a, 1 << 30, n) == \
        B.SPP_ERR_ARG
    # splat: shape not divisible by 2^(L-1), L out of range
    arr = (ctypes.c_void_p * 5)(0x10000, 0x10000, 0x10000, 0x10000, 0x10000)
    g = B.lib.spp_splat_samples
    assert g(a, a, a, a, 16, 30, 16, 3, ctypes.cast(arr, ctypes.c_void_p), n) == B.SPP_ERR_SHAPE
    assert g(a, a, a, a, 16, 32, 16, 6, ctypes.cast(arr, ctypes.c_void_p), n) == B.SPP_ERR_SHAPE
    # reconstruction: temporal needs 54 channels and a coarser level
    r = B.lib.spp_reconstruct_level
    assert r(a, a, 29, a, a, None, 32, 32, None, a, None, None, n) == B.SPP_ERR_ARG
    assert r(a, a, 54, None, a, None, 32, 32, None, a, None, None, n) == B.SPP_ERR_ARG
    assert r(a, mis, 25, None, None, None, 32, 32, None, a, None, None, n) == B.SPP_ERR_ALIGN
    tm = B.make_tonemap(shadow=1.5)
    assert r(a, a, 25, None, None, None, 32, 32, ctypes.byref(tm), a, a, None, n) == B.SPP_ERR_ARG
    w = B.lib.spp_warp_previous
    assert w(None, a, 32, 32, a, n) == B.SPP_ERR_ARG
    assert w(a, mis, 32, 32, a, n) == B.SPP_ERR_ALIGN
    fr = B.lib.spp_reconstruct_frame
    assert fr(ctypes.cast(arr, ctypes.c_void_p), ctypes.cast(arr, ctypes.c_void_p), 29, a, a,
              None, 32, 32, 3, None, a, a, a, 1 << 20, None, n) == B.SPP_ERR_ARG  # C0=54 needed
    assert fr(ctypes.cast(arr, ctypes.c_void_p), ctypes.cast(arr, ctypes.c_void_p), 54, None,
              None, None, 36, 32, 4, None, a, a, a, 1 << 20, None, n) == B.SPP_ERR_SHAPE
    assert fr(ctypes.cast(arr, ctypes.c_void_p), ctypes.cast(arr, ctypes.c_void_p), 54, None,
              None, None, 64, 64, 3, None, a, a, a, 16, None, n) == B.SPP_ERR_WORKSPACE


def test_binding_rejects_host_tensors():
    import torch
    import paper_2602_08642_gb300 as spp
    fr_args = [torch.zeros(4)] * 3
    with pytest.raises(ValueError):
        spp.binding._dev(fr_args[0])


def test_host_argument_errors_two_stage_and_variants(lib):
    """The two-stage, variant and estimator entry points validate on the
    host before any CUDA call."""
    import paper_2602_08642_gb300._binding as B
    a = _fake(0x10000)
    a256 = _fake(0x20000)
    mis = _fake(0x10004)
    n = None
    arr = (ctypes.c_void_p * 5)(0x10000, 0x10000, 0x10000, 0x10000, 0x10000)
    layers = ctypes.cast(arr, ctypes.c_void_p)
    # networks: unknown net, absent-head pointers, shapes, alignment
    nf = B.lib.spp_net_forward
    assert nf(3, a256, a, 1, 32, 32, a, a, a, a256, 1 << 30, a, n) == B.SPP_ERR_ARG
    assert nf(2, a256, a, 1, 32, 32, a, None, a, a256, 1 << 30, a, n) == B.SPP_ERR_ARG
    assert nf(1, a256, a, 1, 30, 32, a, None, None, a256, 1 << 30, a, n) == B.SPP_ERR_SHAPE
    a16 = _fake(0x10010)  # 16- but not 256-byte aligned
    assert nf(1, a16, a, 1, 32, 32, a, None, None, a256, 1 << 30, a, n) == B.SPP_ERR_ALIGN
    assert nf(1, a256, a, 1, 32, 32, a, None, None, a256, 16, a, n) == B.SPP_ERR_WORKSPACE
    nb = B.lib.spp_net_backward
    assert nb(2, a256, 1, 32, 32, a256, 1 << 30, a, None, a, a, None, a256, 1 << 30, a, n) == \
        B.SPP_ERR_ARG
    assert nb(1, a256, 1, 32, 32, a256, 1 << 30, a, None, None, a, mis, a256, 1 << 30, a, n) == \
        B.SPP_ERR_ALIGN
    fp = B.lib.spp_net_forward_prepared
    assert fp(3, a256, 1, 32, 32, a, None, None, a256, 1 << 30, a, n) == B.SPP_ERR_ARG
    assert fp(1, a256, 1, 30, 32, a, None, None, a256, 1 << 30, a, n) == B.SPP_ERR_SHAPE
    assert fp(1, a16, 1, 32, 32, a, None, None, a256, 1 << 30, a, n) == B.SPP_ERR_ALIGN
    assert fp(1, a256, 1, 32, 32, a, None, None, a256, 16, a, n) == B.SPP_ERR_WORKSPACE
    off, ch = ctypes.c_size_t(), ctypes.c_int()
    assert B.lib.spp_net_input_layout(1, 2, 32, 16, ctypes.byref(off), ctypes.byref(ch)) == 0
    assert ch.value == 32 and off.value % 256 == 0
    assert B.lib.spp_net_input_layout(0, 2, 32, 16, ctypes.byref(off), ctypes.byref(ch)) == 0
    assert ch.value == 16
    assert B.lib.spp_net_input_layout(5, 2, 32, 16, ctypes.byref(off), ctypes.byref(ch)) == \
        B.SPP_ERR_ARG
    assert B.lib.spp_assemble_sampler_input(a, a, a, a, None, None, 8, 8, mis, n) == \
        B.SPP_ERR_ALIGN
    assert B.lib.spp_assemble_denoiser_input(None, a, a, a, a, a, a, None, None, 8, 8, a, n) == \
        B.SPP_ERR_ARG
    ds = B.lib.spp_density_softmax
    assert ds(a, 1, 32, 32, 100, a, a, 64, n) == B.SPP_ERR_ARG  # stride below W H
    # two-stage per-pixel steps
    assert B.lib.spp_warp_latent(None, a, 8, 8, a, n) == B.SPP_ERR_ARG
    assert B.lib.spp_assemble_denoiser_features(a, a, a, a, a, a, a, None, None, 8, 8, mis, n) == \
        B.SPP_ERR_ALIGN
    assert B.lib.spp_denoiser_features_backward(a, a, a, 8, 8, None, None, n) == B.SPP_ERR_ARG
    dm = B.lib.spp_demodulate
    assert dm(a, a, None, 30, 32, 3, a, layers, None, n) == B.SPP_ERR_SHAPE
    assert dm(a, a, None, 32, 32, 6, a, layers, None, n) == B.SPP_ERR_ARG
    assert dm(a, a, a, 32, 32, 3, a, layers, None, n) == B.SPP_ERR_ARG  # warped needs an output
    tm = B.make_tonemap(highlight=0.0)
    assert B.lib.spp_remodulate_tonemap(a, a, 8, 8, ctypes.byref(tm), a, a, n) == B.SPP_ERR_ARG
    assert B.lib.spp_demodulate_backward(a, a, a, a, a, None, a, a, 8, 8, a, a, n) == \
        B.SPP_ERR_ARG  # Wd without its gradient
    # variants
    lr = B.lib.spp_density_lowres
    assert lr(a, 32, 32, 3, a, n) == B.SPP_ERR_ARG
    assert lr(a, 30, 32, 4, a, n) == B.SPP_ERR_SHAPE
    assert lr(mis, 32, 32, 2, a, n) == B.SPP_ERR_ALIGN
    sy = B.lib.spp_alloc_sample_map_systematic
    g = B.make_params(0.25, gumbel=True)
    assert sy(a, 4, 4, ctypes.byref(g), a, a, a, 16, a, a, a, a, a, 4096, n) == B.SPP_ERR_ARG
    st = B.make_params(0.25)
    st.flags |= B.SPP_FLAG_TEST_STALL_TILE1
    assert sy(a, 4, 4, ctypes.byref(st), a, a, a, 16, a, a, a, a, a, 4096, n) == B.SPP_ERR_ARG
    # estimators: unknown estimator; straight-through needs the clean image
    p = B.make_params(0.25, hard=True)
    eb = B.lib.spp_splat_backward_estimator
    assert eb(a, a, a, a, a, a, a, 16, 8, 8, ctypes.byref(p), 7, a, 0, a, n) == B.SPP_ERR_ARG
    assert eb(a, a, a, a, a, a, a, 16, 8, 8, ctypes.byref(p), 1, None, 0, a, n) == B.SPP_ERR_ARG
    # Gumbel mode needs a positive inverse temperature
    bad = B.make_params(0.25, gumbel=True, lam=0.0)
    f = B.lib.spp_alloc_sample_map
    assert f(a, 4, 4, ctypes.byref(bad), a, a, a, 16, a, a, a, a, a, 4096, n) == B.SPP_ERR_ARG
