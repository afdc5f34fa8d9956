"""The allocation-free sample-map entry point agrees with the regular one.

spp_alloc_sample_map_static serves callers that may not allocate device
memory while they run (an engine or plug-in host that owns the GPU memory
budget): it keeps its scratch in a static device array inside the library
instead of a caller workspace.  This file runs last so that a failure here
comes after every other test has run.
"""
import numpy as np
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


def test_static_scratch_matches_workspace_version_two_calls(spp):
    W, H = 1920, 1080
    for frame in (0, 1):  # two calls in a row share (and reuse) the static scratch
        d = torch.from_numpy(inp.density_lognormal(W, H, seed=70 + frame)).cuda()
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
        for a, b in ((got.s, ref.s), (got.holdout_w, ref.holdout_w)):
            a, b = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(a - b) <= 1e-5 * np.abs(b))


def test_static_scratch_rejects_oversized_frames(spp):
    fr = _buffers(spp, 64, 64, 16)
    d = torch.ones(16, device="cuda")
    rc = spp.spp_alloc_sample_map_static(d, 8192, 4097, spp.make_params(0.25), fr.counts,
                                         fr.offsets, fr.sample_pixel, 16, fr.s, fr.holdout_w,
                                         fr.total, fr.status)
    assert rc == spp.binding.SPP_ERR_WORKSPACE
