"""Pins of the training-objective oracle (oracle/loss.py) against closed
forms and finite differences."""
import numpy as np

import oracle.loss as L


def test_identical_histories_reduce_to_scaled_l1():
    """With the warped previous output equal to the warped previous
    reference, dI - dI_ref = I - I_ref, so the temporal term 1.25 |I - I_ref|
    wins everywhere: L = 1.25 mean |I - I_ref|."""
    rng = np.random.default_rng(1)
    I, R, P = rng.random((3, 5, 7)), rng.random((3, 5, 7)), rng.random((3, 5, 7))
    loss, g = L.combined_loss(I, R, P, P)
    assert abs(loss - 1.25 * np.abs(I - R).mean()) < 1e-15
    assert np.allclose(g, 1.25 * np.sign(I - R) / I.size)


def test_consistent_motion_reduces_to_l1():
    """When the output changes exactly like the reference (dI = dI_ref) the
    temporal term vanishes and L is the spatial L1."""
    rng = np.random.default_rng(2)
    I, R = rng.random(40), rng.random(40)
    P = rng.random(40)
    loss, g = L.combined_loss(I, R, P, P + (R - I))
    assert abs(loss - np.abs(I - R).mean()) < 1e-15
    assert np.allclose(g, np.sign(I - R) / 40)


def test_gradient_matches_fd_away_from_kinks():
    rng = np.random.default_rng(3)
    n = 60
    I, R, P, Q = rng.random(n), rng.random(n), rng.random(n), rng.random(n)
    _, g = L.combined_loss(I, R, P, Q)
    eps = 1e-7
    s = np.abs(I - R)
    t = 1.25 * np.abs((I - P) - (R - Q))
    for i in range(n):
        if abs(t[i] - s[i]) < 1e-4 or abs(I[i] - R[i]) < 1e-4 or abs((I[i] - P[i]) - (R[i] - Q[i])) < 1e-4:
            continue
        Ip, Im = I.copy(), I.copy()
        Ip[i] += eps
        Im[i] -= eps
        fd = (L.combined_loss(Ip, R, P, Q)[0] - L.combined_loss(Im, R, P, Q)[0]) / (2 * eps)
        assert abs(fd - g[i]) < 1e-8, (i, fd, g[i])


def test_cosine_schedule_endpoints():
    assert L.cosine_lr(0, 100, 1e-3) == 1e-3
    assert abs(L.cosine_lr(50, 100, 1e-3) - 0.5e-3) < 1e-18
    assert abs(L.cosine_lr(100, 100, 1e-3, 1e-5) - 1e-5) < 1e-18


def test_zero_spatial_weight_gives_temporal_l1():
    rng = np.random.default_rng(4)
    I, R, P, Q = (rng.random(30) for _ in range(4))
    loss, _ = L.combined_loss(I, R, P, Q, temporal_weight=1.0, spatial_weight=0.0)
    assert abs(loss - np.abs((I - P) - (R - Q)).mean()) < 1e-15
