"""torch.autograd.Function wrappers of the differentiable steps.

Forward and backward both run in the library's kernels (``libspp.so``);
these classes only allocate the output and gradient tensors and chain the
calls in the order of the chain rule:

    z --DensityToS--> s --Splat--> L^0..L^{L-1} --Reconstruct--> HDR, sRGB --L1Loss--> loss
                                          logits ----^

The discrete sampling decisions (counts, the sample list, the samples
themselves) are held fixed inside a step, as in the paper's relaxed
estimator (Sec. 4.3): gradients reach s through the 1/s normalisation and
the ramp weight, and reach the sampler logits z through the spatial softmax.
"""
from __future__ import annotations

import torch

from . import _binding as B


def _z(t: torch.Tensor) -> torch.Tensor:
    return torch.zeros_like(t)


class Reconstruct(torch.autograd.Function):
    """Coarse-to-fine gather pyramid (Appendix A) with the tone map of Sec. 5.

    apply(L, tm, prev_warp, mask, *layers, *logits) -> (hdr, ldr)
    prev_warp: W_t L_{t-1} at full resolution (spp_warp_previous) or None.
    """

    @staticmethod
    def forward(ctx, L, tm, warped, mask, *tensors):
        layers, logits = list(tensors[:L]), list(tensors[L:2 * L])
        _, H, W = layers[0].shape
        hats = [None] * L
        for l in range(L - 1, 0, -1):
            hats[l] = torch.empty_like(layers[l])
            B.check(B.spp_reconstruct_level(layers[l], logits[l], logits[l].shape[0],
                                            hats[l + 1] if l + 1 < L else None, None, None,
                                            W >> l, H >> l, None, hats[l], None), "level")
        hdr = torch.empty_like(layers[0])
        ldr = torch.empty_like(layers[0])
        B.check(B.spp_reconstruct_level(layers[0], logits[0], logits[0].shape[0], hats[1], warped,
                                        mask if warped is not None else None, W, H, tm, hdr, ldr),
                "level 0")
        ctx.L, ctx.tm = L, tm
        ctx.save_for_backward(warped if warped is not None else torch.empty(0, device=hdr.device),
                              mask if mask is not None else torch.empty(0, device=hdr.device,
                                                                        dtype=torch.uint8),
                              hdr, *layers, *logits, *hats[1:])
        ctx.has_warped = warped is not None
        ctx.has_mask = mask is not None
        return hdr, ldr

    @staticmethod
    def backward(ctx, g_hdr, g_ldr):
        L = ctx.L
        saved = ctx.saved_tensors
        warped = saved[0] if ctx.has_warped else None
        mask = saved[1] if ctx.has_mask else None
        hdr = saved[2]
        layers = list(saved[3:3 + L])
        logits = list(saved[3 + L:3 + 2 * L])
        hats = [None] + list(saved[3 + 2 * L:])
        _, H, W = hdr.shape
        g = torch.zeros_like(hdr) if g_hdr is None else g_hdr.contiguous().clone()
        if g_ldr is not None:
            B.check(B.spp_tonemap_backward(hdr, W, H, ctx.tm, g_ldr.contiguous(), g),
                    "tonemap backward")
        g_layers = [_z(x) for x in layers]
        g_logits = [torch.empty_like(x) for x in logits]
        g_warped = _z(hdr) if warped is not None else None
        for l in range(L):
            g_coarse = _z(hats[l + 1]) if l + 1 < L else None
            B.check(B.spp_reconstruct_level_backward(
                layers[l], logits[l], logits[l].shape[0], hats[l + 1] if l + 1 < L else None,
                warped if l == 0 else None, mask if l == 0 else None, W >> l, H >> l, g,
                g_logits[l], g_layers[l], g_coarse, g_warped if l == 0 else None),
                "level backward")
            g = g_coarse
        return (None, None, g_warped, None, *g_layers, *g_logits)


class WarpPrevious(torch.autograd.Function):
    """W_t L_{t-1} (App. A, Eq. app-recon-full)."""

    @staticmethod
    def forward(ctx, prev, mv):
        _, H, W = prev.shape
        out = torch.empty_like(prev)
        B.check(B.spp_warp_previous(prev, mv, W, H, out), "warp")
        ctx.save_for_backward(mv)
        return out

    @staticmethod
    def backward(ctx, g):
        (mv,) = ctx.saved_tensors
        _, H, W = g.shape
        gp = torch.zeros_like(g)
        B.check(B.spp_warp_previous_backward(mv, W, H, g.contiguous(), gp), "warp backward")
        return gp, None


class L1Loss(torch.autograd.Function):
    """Mean |ldr - ref| (Eq. loss_spatial with the masking term m = 1)."""

    @staticmethod
    def forward(ctx, ldr, ref):
        loss = torch.zeros(4, device=ldr.device)[:1]
        grad = torch.empty_like(ldr)
        B.check(B.spp_l1_loss(ldr, ref, ldr.numel(), loss, grad), "l1")
        ctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None


class Splat(torch.autograd.Function):
    """The noisy pyramid as a function of the density s (Eq. stoch_rnoisy,
    Eq. app-pyramid), the samples and discrete choices of ``frame`` fixed.

    apply(frame, params, s) -> tuple of L layers (those computed by the last
    frame.splat() call)."""

    @staticmethod
    def forward(ctx, frame, params, s):
        ctx.frame, ctx.params, ctx.s_shape = frame, params, s.shape
        return tuple(x.clone() for x in frame.layers)

    @staticmethod
    def backward(ctx, *g_layers):
        fr, p = ctx.frame, ctx.params
        g0 = (g_layers[0].contiguous().clone() if g_layers[0] is not None
              else torch.zeros_like(fr.layers[0]))
        full = [g if g is not None else torch.zeros_like(x) for g, x in zip(g_layers, fr.layers)]
        full = [x.contiguous() for x in full]
        B.check(B.spp_pyramid_backward(full, fr.W, fr.H, fr.L, g0), "pyramid backward")
        gs = torch.empty_like(fr.s)
        B.check(B.spp_splat_backward(fr.offsets, fr.counts, fr.rgb, fr.s, fr.layers[0], g0,
                                     fr.capacity, fr.W, fr.H, p, gs), "splat backward")
        return None, None, gs.view(ctx.s_shape)


class DensityToS(torch.autograd.Function):
    """s = phi B + (1 - phi) B N softmax(z) (Sec. 3), given d = exp(z - max z).

    apply(d, s, budget, phi, z) -> s (the tensor the allocation wrote)."""

    @staticmethod
    def forward(ctx, d, s, budget, phi, z):
        ctx.save_for_backward(d)
        ctx.budget, ctx.phi = budget, phi
        return s.view_as(z).clone()

    @staticmethod
    def backward(ctx, g):
        (d,) = ctx.saved_tensors
        gz = torch.empty_like(d)
        ws = torch.empty(max(B.spp_density_backward_workspace_bytes(), 16), dtype=torch.uint8,
                         device=d.device)
        B.check(B.spp_density_backward(d, d.numel(), ctx.budget, ctx.phi, g.contiguous(), gz, ws),
                "density backward")
        return None, None, None, None, gz.view_as(g)
