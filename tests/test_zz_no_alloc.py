"""The allocation-free sample-map entry point agrees with the regular one.

spp_alloc_sample_map_static serves callers that may not allocate device
memory while they run (an engine or plug-in host that owns the GPU memory
budget): it keeps its scratch in a static device array inside the library
instead of a caller workspace.  Both entry points run the same kernels on
the same inputs, so every output must be bitwise identical.  This file runs
last so that a failure here comes after every other test has run.
"""
import pytest
import torch

import spp_inputs as inp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spp():
    from conftest import build_spp_lib
    build_spp_lib()
    import paper_2602_08642_gb300 as spp
    torch.cuda.set_device(0)
    return spp


def _buffers(spp, W, H, cap):
    fr = spp.Frame(W, H, 1, capacity=cap)
    fr.sample_pixel.fill_(-1)
    fr.clear_status()
    return fr


def _compare(spp, W, H, seed, frame):
    """One call of each entry point on the same density, outputs compared
    bit for bit."""
    d = torch.from_numpy(inp.density_lognormal(W, H, seed=seed)).cuda()
    params = spp.make_params(0.25, frame=frame)
    cap = spp.default_capacity(W, H, 0.25)
    ref = _buffers(spp, W, H, cap)
    ref.alloc(d, params)
    got = _buffers(spp, W, H, cap)
    spp.check(spp.spp_alloc_sample_map_static(
        d, W, H, params, got.counts, got.offsets, got.sample_pixel, cap, got.s,
        got.holdout_w, got.total, got.status), "spp_alloc_sample_map_static")
    torch.cuda.synchronize()
    assert got.check_status() == 0 and ref.check_status() == 0
    T = ref.sample_count()
    assert got.sample_count() == T
    assert torch.equal(got.counts, ref.counts)
    assert torch.equal(got.offsets, ref.offsets)
    assert torch.equal(got.sample_pixel[:T], ref.sample_pixel[:T])
    assert torch.equal(got.s, ref.s)
    assert torch.equal(got.holdout_w, ref.holdout_w)


def test_static_scratch_matches_workspace_version_two_calls(spp):
    for frame in (0, 1):  # two calls in a row share (and reuse) the static scratch
        _compare(spp, 1920, 1080, seed=70 + frame, frame=frame)


def test_static_scratch_sequence_of_sizes(spp):
    """Small frames (few tiles), a 1080p frame, small again and a frame of
    the maximum size, one after the other on one stream: state a call
    leaves in the shared scratch must not reach the next one."""
    for k, (W, H) in enumerate([(128, 128), (1920, 1080), (128, 128), (8192, 4096)]):
        _compare(spp, W, H, seed=80 + k, frame=k)


def test_static_scratch_rejects_oversized_frames(spp):
    fr = _buffers(spp, 64, 64, 16)
    d = torch.ones(16, device="cuda")
    rc = spp.spp_alloc_sample_map_static(d, 8192, 4097, spp.make_params(0.25), fr.counts,
                                         fr.offsets, fr.sample_pixel, 16, fr.s, fr.holdout_w,
                                         fr.total, fr.status)
    assert rc == spp.binding.SPP_ERR_WORKSPACE
