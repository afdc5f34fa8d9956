"""Per-frame driver of the plain method over the C ABI.

Holds the device buffers of one W x H frame (PyTorch allocates them; the
library allocates nothing) and runs the steps of the hot path in order:
sample-count map and sample list, renderer stand-in, splat + pyramid,
coarse-to-fine reconstruction with the temporal term and the tone map.
Every step is a call into ``libspp.so``; this module only sizes buffers and
passes pointers.
"""
from __future__ import annotations

import math

import torch

from . import _binding as B


def logit_channels(level: int, L: int, temporal: bool) -> int:
    if level == L - 1:
        return 25
    if level == 0 and temporal:
        return 54
    return 29


def default_capacity(W: int, H: int, max_budget: float) -> int:
    """Sample slots for a frame: the budget plus a wide statistical margin
    (T is a sum of independent Bernoulli draws around B N)."""
    N = W * H
    return int(max_budget * N + 8.0 * math.sqrt(max(N, 1)) + 4096)


class Frame:
    """Device buffers for W x H frames with an L-level pyramid."""

    def __init__(self, W: int, H: int, L: int, *, max_budget: float = 0.5,
                 capacity: int | None = None, device: str | torch.device = "cuda"):
        self.W, self.H, self.L = W, H, L
        self.N = N = W * H
        self.device = torch.device(device)
        dev = self.device
        self.capacity = capacity if capacity is not None else default_capacity(W, H, max_budget)
        i32, f32 = torch.int32, torch.float32
        self.counts = torch.empty(N, dtype=i32, device=dev)
        self.offsets = torch.empty(N + 1, dtype=i32, device=dev)
        self.sample_pixel = torch.empty(max(self.capacity, 1), dtype=i32, device=dev)
        self.s = torch.empty(N, dtype=f32, device=dev)
        self.holdout_w = torch.empty(N, dtype=f32, device=dev)
        self.total = torch.zeros(2, dtype=torch.int64, device=dev)[:1]
        self.status = torch.zeros(4, dtype=i32, device=dev)[:1]
        self.alloc_ws = torch.empty(max(B.spp_alloc_workspace_bytes(W, H), 16),
                                    dtype=torch.uint8, device=dev)
        self.rgb = torch.empty((max(self.capacity, 1), 4), dtype=f32, device=dev)
        self.layers = [torch.empty((3, H >> l, W >> l), dtype=f32, device=dev) for l in range(L)]
        self.recon_ws = torch.empty(max(B.spp_reconstruct_workspace_bytes(W, H, L), 16),
                                    dtype=torch.uint8, device=dev)
        self.hdr = [torch.zeros((3, H, W), dtype=f32, device=dev) for _ in range(2)]
        self.ldr = torch.empty((3, H, W), dtype=f32, device=dev)
        self.parity = 0  # which hdr buffer receives the next output

    # ----------------------------------------------------------------- steps
    def alloc(self, d: torch.Tensor, params: B.spp_params, stream=None):
        B.check(B.spp_alloc_sample_map(d, self.W, self.H, params, self.counts, self.offsets,
                                       self.sample_pixel, self.capacity, self.s, self.holdout_w,
                                       self.total, self.status, self.alloc_ws, stream),
                "spp_alloc_sample_map")

    def alloc_dithered(self, d: torch.Tensor, params: B.spp_params, mask: torch.Tensor,
                       stream=None):
        """alloc with the uniforms from a blue-noise rank mask (device int16
        view of spp_blue_noise_mask's uint16 [T][T])."""
        B.check(B.spp_alloc_sample_map_dithered(d, self.W, self.H, params, mask, self.counts,
                                                self.offsets, self.sample_pixel, self.capacity,
                                                self.s, self.holdout_w, self.total, self.status,
                                                self.alloc_ws, stream),
                "spp_alloc_sample_map_dithered")

    def alloc_systematic(self, d: torch.Tensor, params: B.spp_params, stream=None):
        """alloc with systematic (exact-integer-total) rounding."""
        B.check(B.spp_alloc_sample_map_systematic(d, self.W, self.H, params, self.counts,
                                                  self.offsets, self.sample_pixel, self.capacity,
                                                  self.s, self.holdout_w, self.total,
                                                  self.status, self.alloc_ws, stream),
                "spp_alloc_sample_map_systematic")

    def render(self, clean: torch.Tensor, seed: int, frame: int, stream=None):
        B.check(B.spp_render_synthetic(clean, self.offsets, self.sample_pixel, self.total,
                                       self.capacity, self.W, self.H, seed, frame, self.rgb,
                                       stream), "spp_render_synthetic")

    def splat(self, stream=None):
        B.check(B.spp_splat_samples(self.offsets, self.rgb, self.s, self.holdout_w,
                                    self.capacity, self.W, self.H, self.L, self.layers, stream),
                "spp_splat_samples")

    def reconstruct(self, logits, prev=None, mv=None, mask=None, tm=None, stream=None):
        out = self.hdr[self.parity]
        C0 = logits[0].shape[0]
        B.check(B.spp_reconstruct_frame(self.layers, logits, C0, prev, mv, mask, self.W, self.H,
                                        self.L, tm if tm is not None else B.make_tonemap(), out,
                                        self.ldr, self.recon_ws, self.status, stream),
                "spp_reconstruct_frame")
        self.parity ^= 1
        return out

    def run(self, d, clean, logits, params: B.spp_params, *, render_seed: int = 0xC0FFEE,
            prev=None, mv=None, mask=None, tm=None, stream=None):
        """One frame of the plain method; returns the HDR output tensor."""
        self.alloc(d, params, stream)
        self.render(clean, render_seed, params.frame, stream)
        self.splat(stream)
        return self.reconstruct(logits, prev=prev, mv=mv, mask=mask, tm=tm, stream=stream)

    def check_status(self, stream=None) -> int:
        code = B.spp_get_status(self.status, stream)
        B.check(code, "device status")
        return code

    def clear_status(self, stream=None):
        B.check(B.spp_clear_status(self.status, stream), "spp_clear_status")

    def sample_count(self) -> int:
        return int(self.total.item())
