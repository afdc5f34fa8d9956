"""The two-stage pipeline of Sec. 3 (sampler network before rendering,
denoiser network after it, shared recurrent latents) with the learned
demodulation of Sec. 6.2, and its training loop, driven over the C ABI.

One frame t of sample b:
  warp    W_t of the previous HDR output, its tone map (the sampler's
          recurrent input) and W_t tanh of the previous denoiser's latents
  sampler G-buffer + warped LDR + warped latents -> density logit z ->
          d = exp(z - max z)
  render  stochastic rounding of s (Sec. 4), renderer stand-in, splat -> L^0
  denoiser ln(1+L^0), ln(1+s), ln(1+n), G-buffer, ln(1 + W_t L_{t-1}),
          warped latents -> 54 / 29 / 25 kernel logits, demodulation
          channels c, raw latents
  reconstruct  m = exp(clamp(c)); gather pyramid on pyr(L^0 / m) with the
          temporal term over W_t L_{t-1} / m; out = m * R; tone map

Training (two-frame window, like the joint predictor's): frame t-1 runs
forward only and provides the recurrent inputs of frame t; the loss of frame
t is back-propagated through the tone map, the remodulation, the gather
pyramid, the demodulation, the denoiser (into its parameters and its input),
the splat (through 1/s and the relaxed holdout ramp, Sec. 4.3), the spatial
softmax and the sampler.  The latents passed between frames are held
constant (no back-propagation through time).  Every step is a library call;
this module allocates buffers and orders the calls.
"""
from __future__ import annotations

import math

import torch

from . import _binding as B
from .learned import LEVELS, PHI, Predictor, random_tonemap
from .pipeline import Frame

NL = B.SPP_LATENT_CHANNELS
DP = B.SPP_DEMOD_PLANE
LP = B.SPP_LATENT_PLANE


def _zeros(*shape, dtype=torch.float32):
    return torch.zeros(*shape, dtype=dtype, device="cuda")


def layer_table(net: int):
    """[(name, cin, cout, relu)] of the present layers of network `net`, in
    parameter order (from the library)."""
    names = ("e0a", "e0b", "e1a", "e1b", "e2a", "e2b", "h2", "d1a", "d1b", "h1", "d0a", "d0b",
             "h0")
    out = []
    for i, n in enumerate(names):
        cin, cout, relu = B.spp_net_layer(net, i)
        if cout:
            out.append((n, cin, cout, relu))
    return out


def flops_per_frame(W: int, H: int) -> int:
    """Multiply-adds x 2 of one sampler and one denoiser forward pass."""
    total = 0
    for net in (B.SPP_NET_SAMPLER, B.SPP_NET_DENOISER):
        for i in range(13):
            cin, cout, _ = B.spp_net_layer(net, i)
            lv = (0, 0, 1, 1, 2, 2, 2, 1, 1, 1, 0, 0, 0)[i]
            total += 2 * 9 * cin * cout * (W >> lv) * (H >> lv)
    return total


class TwoStage:
    """Sampler + denoiser state for batches of B frames of W x H."""

    def __init__(self, theta_s: torch.Tensor, theta_d: torch.Tensor, B_: int, W: int, H: int,
                 budget: float, train: bool = False, dither_mask=None, density_factor: int = 1,
                 rounding: str = "stochastic"):
        """density_factor > 1 samples from the density averaged over
        factor x factor blocks (the low-resolution density map of Sec. 7);
        rounding "systematic" uses the exact-integer-total sample map
        (inference only: the splat's backward recomputes the white-noise
        uniforms of the stochastic map)."""
        if rounding not in ("stochastic", "systematic"):
            raise ValueError("rounding must be 'stochastic' or 'systematic'")
        if rounding == "systematic" and (train or dither_mask is not None):
            raise ValueError("systematic rounding is an inference-time variant")
        self.B, self.W, self.H, self.budget, self.train = B_, W, H, budget, train
        self.density_factor, self.rounding = density_factor, rounding
        self.d_lr = [_zeros(H, W) for _ in range(B_)] if density_factor > 1 else None
        self.sampler = Predictor(theta_s, B_, W, H, train, net=B.SPP_NET_SAMPLER)
        self.denoiser = Predictor(theta_d, B_, W, H, train, net=B.SPP_NET_DENOISER,
                                  input_grad=train)
        # the assembly kernels write each network's BF16 NHWC input in place
        self.sp_in = [self.sampler.input_nhwc(b) for b in range(B_)]
        self.dn_in = [self.denoiser.input_nhwc(b) for b in range(B_)]
        self.dither = dither_mask
        self.tm = B.make_tonemap()
        self.frames = [Frame(W, H, LEVELS, max_budget=budget) for _ in range(B_)]
        z3 = lambda: [_zeros(3, H, W) for _ in range(B_)]
        self.hdr_prev, self.warped, self.warped_ldr = z3(), z3(), z3()
        self.latent = [_zeros(NL, H, W) for _ in range(B_)]  # tanh of the raw planes
        self.warped_latent = [_zeros(NL, H, W) for _ in range(B_)]
        self.m, self.wd, self.hdr, self.ldr = z3(), z3(), z3(), z3()
        self.dlayers = [[_zeros(3, H >> l, W >> l) for l in range(LEVELS)] for _ in range(B_)]
        self.hats = [[_zeros(3, H >> l, W >> l) for l in range(LEVELS)] for _ in range(B_)]
        self.mask = _zeros(H, W, dtype=torch.uint8)
        self.has_prev = False
        self.cur_temporal = False
        self.params = [None] * B_
        self.ref = z3()
        self.loss = [_zeros(4)[:1] for _ in range(B_)]
        self.mse = torch.zeros(2, dtype=torch.float64, device="cuda")[:1]
        if train:
            self.g_ldr = _zeros(3, H, W)
            self.g_out = _zeros(3, H, W)
            self.g_R = [_zeros(3, H >> l, W >> l) for l in range(LEVELS)]
            self.g_noisy = [_zeros(3, H >> l, W >> l) for l in range(LEVELS)]
            self.g_wd = _zeros(3, H, W)
            self.g_L0 = z3()
            self.g_s = _zeros(W * H)
            self.dbws = Predictor._aligned(B.spp_density_backward_workspace_bytes())
            self.ldr_prev, self.wldr_prev, self.wref_prev, self.tmp = z3(), z3(), z3(), z3()

    def begin_sequence(self):
        self.has_prev = False

    def _alloc(self, b, fr, d, params):
        if self.density_factor > 1:
            B.check(B.spp_density_lowres(d, self.W, self.H, self.density_factor, self.d_lr[b]),
                    "density lowres")
            d = self.d_lr[b]
        if self.dither is not None:
            fr.alloc_dithered(d, params, self.dither)
        elif self.rounding == "systematic":
            fr.alloc_systematic(d, params)
        else:
            fr.alloc(d, params)

    def frame(self, gbufs: list, mvs: list, cleans: list, seed: int, frame_index: int):
        """Forward of one frame of every sample (gbufs[b]: dict of albedo,
        normal, depth; mvs[b]: motion to the previous frame; cleans[b]: the
        clean radiance the renderer stand-in samples)."""
        W, H, L = self.W, self.H, LEVELS
        sp, dn = self.sampler, self.denoiser
        tp = self.has_prev
        self.cur_temporal = tp
        for b in range(self.B):
            if tp:
                B.check(B.spp_warp_previous(self.hdr_prev[b], mvs[b], W, H, self.warped[b]), "warp")
                B.check(B.spp_tonemap_image(self.warped[b], W, H, self.tm, self.warped_ldr[b]),
                        "tonemap")
                B.check(B.spp_warp_channels(self.latent[b], NL, mvs[b], W, H,
                                            self.warped_latent[b]), "warp latent")
            g = gbufs[b]
            B.check(B.spp_assemble_sampler_input(
                g["albedo"], g["normal"], g["depth"], mvs[b], self.warped_ldr[b] if tp else None,
                self.warped_latent[b] if tp else None, W, H, self.sp_in[b]), "sampler input")
        sp.forward_prepared()
        for b in range(self.B):
            fr = self.frames[b]
            self.params[b] = B.make_params(self.budget, uniform_fraction=PHI, seed=seed + b,
                                           frame=frame_index)
            self._alloc(b, fr, sp.density[b], self.params[b])
            fr.render(cleans[b], (seed + b) ^ 0xC0FFEE, frame_index)
            fr.splat()
            g = gbufs[b]
            B.check(B.spp_assemble_denoiser_input(
                fr.layers[0], fr.s, fr.counts, g["albedo"], g["normal"], g["depth"], mvs[b],
                self.warped[b] if tp else None, self.warped_latent[b] if tp else None, W, H,
                self.dn_in[b]), "denoiser input")
        dn.forward_prepared()
        for b in range(self.B):
            fr = self.frames[b]
            h0 = dn.heads[0][b]
            B.check(B.spp_demodulate(fr.layers[0], h0[DP:DP + 3], self.warped[b] if tp else None,
                                     W, H, L, self.m[b], self.dlayers[b],
                                     self.wd[b] if tp else None), "demodulate")
            lg = self.logits(b)
            hats = self.hats[b]
            for l in range(L - 1, -1, -1):
                B.check(B.spp_reconstruct_level(
                    self.dlayers[b][l], lg[l], lg[l].shape[0], hats[l + 1] if l + 1 < L else None,
                    self.wd[b] if (l == 0 and tp) else None, self.mask if (l == 0 and tp) else None,
                    W >> l, H >> l, None, hats[l], None), "reconstruct level")
            B.check(B.spp_remodulate_tonemap(hats[0], self.m[b], W, H, self.tm, self.hdr[b],
                                             self.ldr[b]), "remodulate")
        for b in range(self.B):
            self.hdr_prev[b].copy_(self.hdr[b])
            B.check(B.spp_latent_tanh(dn.heads[0][b, LP:LP + NL], W, H, self.latent[b]),
                    "latents")
        self.has_prev = True

    def logits(self, b: int):
        """Kernel logits of sample b per level (54 planes at level 0 with the
        temporal term, else the first 29)."""
        h = self.denoiser.heads
        n0 = 54 if self.cur_temporal else 29
        return [h[0][b, :n0], h[1][b], h[2][b]]

    def reference(self, b: int, clean):
        B.check(B.spp_tonemap_image(clean, self.W, self.H, self.tm, self.ref[b]), "tonemap")

    def psnr(self, b: int) -> float:
        B.check(B.spp_mse(self.ldr[b], self.ref[b], 3 * self.W * self.H, self.mse), "mse")
        return -10.0 * math.log10(max(float(self.mse.item()), 1e-30))

    # ------------------------------------------------------------ training
    def backward(self, b: int, objective: str = "l1"):
        """Loss of frame b and the head gradients of both networks (the
        denoiser's level-0 head: kernel logits and demodulation channels;
        the sampler's density logit is filled by :meth:`backward_sampler`)."""
        W, H, L = self.W, self.H, LEVELS
        fr, dn = self.frames[b], self.denoiser
        n = 3 * W * H
        if objective == "combined":
            B.check(B.spp_combined_loss(self.ldr[b], self.ref[b], self.wldr_prev[b],
                                        self.wref_prev[b], n, 1.25, 1.0, self.loss[b], self.g_ldr),
                    "combined loss")
        else:
            B.check(B.spp_l1_loss(self.ldr[b], self.ref[b], n, self.loss[b], self.g_ldr), "l1")
        self.g_out.zero_()  # spp_tonemap_backward accumulates
        B.check(B.spp_tonemap_backward(self.hdr[b], W, H, self.tm, self.g_ldr, self.g_out),
                "tonemap backward")
        B.check(B.spp_remodulate_backward(self.g_out, self.m[b], W, H, self.g_R[0]),
                "remodulate backward")
        tp = self.cur_temporal
        lg = self.logits(b)
        gh = dn.g_heads
        g_lg = [gh[0][b, :lg[0].shape[0]], gh[1][b], gh[2][b]]
        gh[0][b].zero_()
        for t in self.g_noisy:
            t.zero_()
        self.g_wd.zero_()
        hats = self.hats[b]
        for l in range(L):
            gc = self.g_R[l + 1] if l + 1 < L else None
            if gc is not None:
                gc.zero_()
            B.check(B.spp_reconstruct_level_backward(
                self.dlayers[b][l], lg[l], lg[l].shape[0], hats[l + 1] if l + 1 < L else None,
                self.wd[b] if (l == 0 and tp) else None, self.mask if (l == 0 and tp) else None,
                W >> l, H >> l, self.g_R[l], g_lg[l], self.g_noisy[l], gc,
                self.g_wd if (l == 0 and tp) else None), "level backward")
        B.check(B.spp_pyramid_backward(self.g_noisy, W, H, L, self.g_noisy[0]), "pyramid backward")
        h0 = dn.heads[0][b]
        B.check(B.spp_demodulate_backward(
            self.hdr[b], self.g_out, self.dlayers[b][0], self.g_noisy[0],
            self.wd[b] if tp else None, self.g_wd if tp else None, h0[DP:DP + 3], self.m[b], W, H,
            self.g_L0[b], gh[0][b, DP:DP + 3]), "demodulate backward")

    def backward_sampler(self, b: int):
        """After the denoiser's backward (its input gradient): the gradient
        of L^0 and s through the denoiser input, the splat and the density."""
        W, H = self.W, self.H
        fr, dn, sp = self.frames[b], self.denoiser, self.sampler
        B.check(B.spp_denoiser_features_backward(fr.layers[0], fr.s, dn.g_x[b], W, H,
                                                 self.g_L0[b], None), "features backward")
        B.check(B.spp_splat_backward(fr.offsets, fr.counts, fr.rgb, fr.s, fr.layers[0],
                                     self.g_L0[b], fr.capacity, W, H, self.params[b], self.g_s),
                "splat backward")
        B.check(B.spp_denoiser_features_backward(fr.layers[0], fr.s, dn.g_x[b], W, H, None,
                                                 self.g_s), "features backward")
        if self.density_factor > 1:  # P is symmetric: the same map on the gradient
            B.check(B.spp_density_lowres(self.g_s, W, H, self.density_factor, self.g_s),
                    "density lowres backward")
        B.check(B.spp_density_backward(sp.density[b], W * H, self.budget, PHI, self.g_s,
                                       sp.g_heads[0][b, 0], self.dbws), "density backward")

    def temporal_references(self, b: int, clean_prev, mv):
        W, H = self.W, self.H
        B.check(B.spp_warp_previous(self.ldr_prev[b], mv, W, H, self.wldr_prev[b]), "warp")
        B.check(B.spp_tonemap_image(clean_prev, W, H, self.tm, self.tmp[b]), "tonemap")
        B.check(B.spp_warp_previous(self.tmp[b], mv, W, H, self.wref_prev[b]), "warp")


class TwoStageTrainer:
    """Trains the sampler and the denoiser jointly on two-frame samples
    (learned.FrameData); options as learned.Trainer, plus density_factor (the
    low-resolution density map)."""

    def __init__(self, theta_s, theta_d, batch: int, size: int, budget: float = 0.25,
                 lr: float = 1e-3, weight_decay: float = 1e-4, objective: str = "l1",
                 betas=(0.9, 0.999), random_tmo: bool = False, total_steps: int | None = None,
                 seed: int = 0, dither_mask=None, density_factor: int = 1):
        import numpy as np
        self.p = TwoStage(theta_s, theta_d, batch, size, size, budget, train=True,
                          dither_mask=dither_mask, density_factor=density_factor)
        self.lr, self.wd = lr, weight_decay
        self.objective, self.betas, self.random_tmo = objective, betas, random_tmo
        self.total_steps = total_steps
        self.rng = np.random.default_rng(seed)
        self.step_index = 0

    def current_lr(self) -> float:
        if not self.total_steps:
            return self.lr
        k = min(self.step_index, self.total_steps)
        return 0.5 * self.lr * (1.0 + math.cos(math.pi * k / self.total_steps))

    def step(self, samples: list, seed: int) -> float:
        p = self.p
        if self.random_tmo:
            p.tm = random_tonemap(self.rng)
        f_prev, f_cur = 2 * self.step_index, 2 * self.step_index + 1
        p.begin_sequence()
        p.frame([s.gprev for s in samples], [s.mv for s in samples],
                [s.clean_prev for s in samples], seed, f_prev)
        if self.objective == "combined":
            for b in range(p.B):
                p.ldr_prev[b].copy_(p.ldr[b])
        p.frame([s.g for s in samples], [s.mv for s in samples], [s.clean for s in samples],
                seed, f_cur)
        for b, s in enumerate(samples):
            p.reference(b, s.clean)
            if self.objective == "combined":
                p.temporal_references(b, s.clean_prev, s.mv)
            p.backward(b, self.objective)
        p.denoiser.backward()
        for b in range(p.B):
            p.backward_sampler(b)
        p.sampler.backward()
        scale = 1.0 / len(samples)
        for net in (p.sampler, p.denoiser):
            net.adamw(self.current_lr(), self.wd, grad_scale=scale, betas=self.betas)
        self.step_index += 1
        return float(sum(l.item() for l in p.loss)) / len(samples)


def evaluate(samples: list, budget: float, theta_s, theta_d, seed: int = 99,
             dither_mask=None, density_factor: int = 1,
             rounding: str = "stochastic") -> list[float]:
    """PSNR of frame t of each two-frame sample (as learned.evaluate)."""
    W, H = samples[0].W, samples[0].H
    p = TwoStage(theta_s, theta_d, 1, W, H, budget, dither_mask=dither_mask,
                 density_factor=density_factor, rounding=rounding)
    out = []
    for i, s in enumerate(samples):
        p.begin_sequence()
        p.frame([s.gprev], [s.mv], [s.clean_prev], seed + i, 0)
        p.frame([s.g], [s.mv], [s.clean], seed + i, 1)
        p.reference(0, s.clean)
        out.append(p.psnr(0))
    return out
