"""FP64 oracle of the training objective of Sec. 6.3 (test infrastructure
only, like the rest of ``oracle/``).

Eq. loss_spatial with the MILO mask m = 1:   S = |I - I_ref|
Eq. loss_temporal:                           T = |dI - dI_ref|,
    dI = I - W(I_prev), dI_ref = I_ref - W(I_ref_prev)
    (tone-mapped sRGB images; W the motion-compensating warp, applied by the
    caller, so the inputs here are the warped previous images)
Eq. loss_combined:                           L = max(1.25 T, S)

Reading: the maximum is taken per element and then averaged over the n
elements (the paper writes the terms per pixel and does not say where the
mean is taken); ties go to the spatial term.  The previous frame is a
constant of the step (two-frame window, the loss on the current frame), so
the gradient with respect to I is, per element,
    1.25 sign(dI - dI_ref) / n   where the temporal term wins,
    sign(I - I_ref) / n          elsewhere.
"""
from __future__ import annotations

import numpy as np


def combined_loss(ldr, ref, prev_warped, ref_prev_warped, temporal_weight: float = 1.25,
                  spatial_weight: float = 1.0):
    """(L, dL/d ldr) in FP64 of mean max(w_t T, w_s S); the paper's weights
    are w_t = 1.25, w_s = 1 (w_s = 0 gives the temporal error alone)."""
    I = np.asarray(ldr, np.float64)
    R = np.asarray(ref, np.float64)
    dI = I - np.asarray(prev_warped, np.float64)
    dR = R - np.asarray(ref_prev_warped, np.float64)
    s = spatial_weight * np.abs(I - R)
    t = temporal_weight * np.abs(dI - dR)
    n = I.size
    temporal = t > s
    loss = float(np.where(temporal, t, s).sum() / n)
    grad = np.where(temporal, temporal_weight * np.sign(dI - dR),
                    spatial_weight * np.sign(I - R)) / n
    return loss, grad


def cosine_lr(step: int, total: int, lr_max: float, lr_min: float = 0.0) -> float:
    """Cosine annealing (Loshchilov & Hutter, SGDR without restarts): the
    learning rate of step 0 <= step < total."""
    return lr_min + 0.5 * (lr_max - lr_min) * (1.0 + np.cos(np.pi * step / max(total, 1)))
