"""The library's blue-noise mask generator (host code, no GPU) against the
oracle's independent implementation of the same published method: equal
rank matrices."""
import numpy as np
import pytest

import oracle.bluenoise as BN


@pytest.fixture(scope="module")
def lib():
    from conftest import build_spp_lib
    build_spp_lib()
    import paper_2602_08642_gb300 as spp
    return spp.binding


@pytest.mark.parametrize("T,seed", [(4, 1), (16, 3), (32, 99), (64, 7), (64, 0x5EED)])
def test_mask_matches_oracle(lib, T, seed):
    assert np.array_equal(lib.spp_blue_noise_mask(T, seed), BN.mask(T, seed))


@pytest.mark.parametrize("T", [0, 3, 12, 512])
def test_mask_rejects_bad_size(lib, T):
    from paper_2602_08642_gb300._binding import SppError
    with pytest.raises(SppError):
        lib.spp_blue_noise_mask(T, 1)
