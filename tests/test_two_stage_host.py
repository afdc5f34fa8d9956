"""Host-side checks of the two-stage pipeline's boundary (no GPU): the
network specifications and layer tables the library reports equal the
oracle's, and invalid arguments are rejected before any launch."""
import pytest

import oracle.unet as U


@pytest.fixture(scope="module")
def B():
    from conftest import build_spp_lib
    build_spp_lib()
    from paper_2602_08642_gb300 import _binding
    return _binding


NETS = {"joint": 0, "sampler": 1, "denoiser": 2}


@pytest.mark.parametrize("spec", sorted(NETS))
def test_specs_and_layer_tables_match_the_oracle(B, spec):
    net = NETS[spec]
    cin, heads = B.spp_net_spec(net)
    assert (cin, heads) == U.SPECS[spec]
    assert B.spp_net_param_count(net) == U.param_offsets(spec)[1]
    table = [B.spp_net_layer(net, i) for i in range(13)]
    present = [(c_in, c_out, bool(relu)) for c_in, c_out, relu in table if c_out > 0]
    assert present == [(ci, co, r) for _, ci, co, r in U.layers(spec)]


def test_invalid_network_arguments(B):
    assert B.spp_net_param_count(3) == -1 and B.spp_net_param_count(-1) == -1
    assert B.spp_net_packed_bytes(7, 0) == 0
    assert B.spp_net_workspace_bytes(1, -1, 8, 8) == 0
    with pytest.raises(B.SppError):
        B.spp_net_spec(5)
    with pytest.raises(B.SppError):
        B.spp_net_layer(1, 13)
    assert B.SPP_DEMOD_PLANE == 54 and B.SPP_LATENT_PLANE == 57 and B.SPP_LATENT_CHANNELS == 7
    assert B.SPP_LATENT_PLANE + B.SPP_LATENT_CHANNELS == U.SPECS["denoiser"][1][0]


@pytest.mark.parametrize("spec", sorted(NETS))
@pytest.mark.parametrize("Bn,W,H", [(1, 32, 32), (2, 48, 36), (8, 128, 128), (1, 3840, 2160)])
def test_input_copy_lies_inside_the_forward_workspace(B, spec, Bn, W, H):
    """The BF16 NHWC input copy the assembly entries write in place: aligned
    for the 16-byte vector stores, padded to 16 or 32 channels, and wholly
    inside the forward workspace."""
    net = NETS[spec]
    off, ch = B.spp_net_input_layout(net, Bn, W, H)
    cin, _ = B.spp_net_spec(net)
    assert ch == (16 if cin <= 16 else 32) and ch >= cin
    assert off % 256 == 0
    assert off + Bn * H * W * ch * 2 <= B.spp_net_workspace_bytes(net, Bn, W, H)
