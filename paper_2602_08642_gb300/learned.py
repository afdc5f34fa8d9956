"""The learned sampler / kernel predictor (Sec. 3, Sec. 6.3) and its
training loop, driven over the C ABI.

Every arithmetic step runs in ``libspp.so``: feature assembly, the tensor-
core U-Net forward and backward, the density softmax and its gradient, the
sampling, splatting and reconstruction with their backward passes, the L1
loss in tone-mapped sRGB, AdamW and the parameter packing.  This module
allocates the buffers (PyTorch) and calls the entry points in order.

One training step (after Sec. 6.3, two-frame window):
  frame t-1  features without a previous output -> network -> density and
             logits -> samples -> reconstruction without the temporal term
  frame t    previous output warped along the motion vectors and tone
             mapped -> features -> network -> samples -> reconstruction with
             the temporal term -> L1 against the tone-mapped reference;
             gradients flow back through the tone map, the reconstruction
             (kernel logits), the splat (density s through 1/s and the
             holdout ramp, Sec. 4.3) and the spatial softmax into the
             network, whose parameters take one AdamW step.
"""
from __future__ import annotations

import math

import torch

from . import _binding as B
from .pipeline import Frame

LEVELS = 3
PHI = 0.125
# names of the network's layers in parameter order (spp_unet_layer gives the shapes)
LAYER_NAMES = ("e0a", "e0b", "e1a", "e1b", "e2a", "e2b", "h2", "d1a", "d1b", "h1", "d0a", "d0b",
               "h0")
LAYER_LEVEL = (0, 0, 1, 1, 2, 2, 2, 1, 1, 1, 0, 0, 0)


def layer_table():
    """[(name, cin, cout, relu)] from the library."""
    return [(n, *B.spp_unet_layer(i)) for i, n in enumerate(LAYER_NAMES)]


def flops_per_frame(W: int, H: int) -> int:
    """Multiply-adds x 2 of one forward pass on a W x H frame (real channel
    counts, zero padding not counted)."""
    total = 0
    for i, (_, cin, cout, _) in enumerate(layer_table()):
        lv = LAYER_LEVEL[i]
        total += 2 * 9 * cin * cout * (W >> lv) * (H >> lv)
    return total


def _zeros(*shape, dtype=torch.float32):
    return torch.zeros(*shape, dtype=dtype, device="cuda")


class Predictor:
    """Device state of one network (the joint predictor by default; the
    sampler or the denoiser of the two-stage pipeline with ``net``) for
    batches of B frames of W x H."""

    def __init__(self, theta: torch.Tensor, B_: int, W: int, H: int, train: bool = False,
                 net: int = B.SPP_NET_JOINT, input_grad: bool = False):
        if W % 4 or H % 4:
            raise ValueError("W and H must be divisible by 4")
        self.B, self.W, self.H, self.train, self.net = B_, W, H, train, net
        self.cin, self.head_ch = B.spp_net_spec(net)
        self.theta = theta.detach().to("cuda", torch.float32).contiguous().clone()
        if self.theta.numel() != B.spp_net_param_count(net):
            raise ValueError("theta has the wrong size")
        self.packed = self._aligned(B.spp_net_packed_bytes(net, train))
        self.fws = self._aligned(B.spp_net_workspace_bytes(net, B_, W, H))
        self.x = _zeros(B_, self.cin, H, W)
        self.heads = [None if c == 0 else _zeros(B_, c, H >> l, W >> l)
                      for l, c in enumerate(self.head_ch)]
        self.density = _zeros(B_, H, W)
        self.dws = self._aligned(B.spp_density_softmax_workspace_bytes(B_))
        self.status = _zeros(4, dtype=torch.int32)[:1]
        if train:
            self.bws = self._aligned(B.spp_net_backward_workspace_bytes(net, B_, W, H))
            self.grad = _zeros(self.theta.numel())
            self.m = _zeros(self.theta.numel())
            self.v = _zeros(self.theta.numel())
            self.g_heads = [None if t is None else torch.zeros_like(t) for t in self.heads]
            self.g_x = torch.zeros_like(self.x) if input_grad else None
            self.step_count = 0
        self.pack()

    # the joint network's names
    @property
    def in12(self):
        return self.x

    @property
    def logits(self):
        return self.heads

    @property
    def g_logits(self):
        return self.g_heads

    @staticmethod
    def _aligned(n: int) -> torch.Tensor:
        buf = torch.empty(int(n) + 256, dtype=torch.uint8, device="cuda")
        off = (-buf.data_ptr()) % 256
        return buf[off:off + int(n)]

    def pack(self):
        B.check(B.spp_net_pack(self.net, self.theta, self.train, self.packed), "spp_net_pack")

    def features(self, b: int, albedo, normal, depth, mv, prev_ldr=None):
        B.check(B.spp_assemble_features(albedo, normal, depth, mv, prev_ldr, self.W, self.H,
                                        self.x[b]), "spp_assemble_features")

    def forward(self):
        if self.net == B.SPP_NET_JOINT:
            B.check(B.spp_predict_density_and_kernels(self.packed, self.x, self.B, self.W, self.H,
                                                      self.density, *self.heads, self.fws,
                                                      self.status), "spp_predict")
            return
        B.check(B.spp_net_forward(self.net, self.packed, self.x, self.B, self.W, self.H,
                                  *self.heads, self.fws, self.status), "spp_net_forward")
        if self.net == B.SPP_NET_SAMPLER:
            hw = self.W * self.H
            B.check(B.spp_density_softmax(self.heads[0], self.B, self.W, self.H, hw, self.density,
                                          self.dws), "spp_density_softmax")

    def input_nhwc(self, b: int) -> torch.Tensor:
        """The forward's BF16 NHWC input copy of image b inside the workspace,
        [H][W][channels]; written by the direct assembly entries, consumed
        by forward_prepared."""
        off, ch = B.spp_net_input_layout(self.net, self.B, self.W, self.H)
        n = self.H * self.W * ch
        return self.fws[off + 2 * n * b: off + 2 * n * (b + 1)].view(torch.bfloat16).view(
            self.H, self.W, ch)

    def forward_prepared(self):
        """Forward on the BF16 input already in the workspace (input_nhwc)."""
        B.check(B.spp_net_forward_prepared(self.net, self.packed, self.B, self.W, self.H,
                                           *self.heads, self.fws, self.status),
                "spp_net_forward_prepared")
        if self.net == B.SPP_NET_SAMPLER:
            hw = self.W * self.H
            B.check(B.spp_density_softmax(self.heads[0], self.B, self.W, self.H, hw, self.density,
                                          self.dws), "spp_density_softmax")

    def backward(self):
        B.check(B.spp_net_backward(self.net, self.packed, self.B, self.W, self.H, self.fws,
                                   *self.g_heads, self.grad, self.g_x, self.bws, self.status),
                "spp_net_backward")

    def adamw(self, lr: float, weight_decay: float = 1e-4, grad_scale: float = 1.0,
              betas=(0.9, 0.999)):
        self.step_count += 1
        B.check(B.spp_adamw_step(self.theta, self.grad, self.m, self.v, self.step_count, lr=lr,
                                 beta1=betas[0], beta2=betas[1], weight_decay=weight_decay,
                                 grad_scale=grad_scale), "adamw")
        self.pack()

    def frame_logits(self, b: int, temporal: bool):
        l0 = self.heads[0][b, :54] if temporal else self.heads[0][b, :29]
        return [l0, self.heads[1][b], self.heads[2][b]]


REF_SPP = 64  # samples per pixel of the rendered references
_REF_FRAMES: dict = {}


def render_reference(clean: torch.Tensor, seed: int, frame: int = 0,
                     spp: int = REF_SPP) -> torch.Tensor:
    """HDR reference of one frame: the mean of `spp` samples per pixel of the
    renderer stand-in (the paper trains against converged renders of each
    frame; this is their synthetic counterpart), rendered by the library's
    own sample map (a uniform density at budget `spp` gives every pixel
    exactly `spp` samples and no extra one), renderer and splat."""
    H, W = clean.shape[1:]
    key = (W, H, spp)
    if key not in _REF_FRAMES:
        _REF_FRAMES.clear()  # one reference size at a time keeps memory bounded
        _REF_FRAMES[key] = (Frame(W, H, 1, max_budget=float(spp), capacity=spp * W * H),
                            torch.ones(H, W, device="cuda"))
    fr, ones = _REF_FRAMES[key]
    fr.alloc(ones, B.make_params(float(spp), uniform_fraction=PHI, seed=seed, frame=frame,
                                 hard=True))
    fr.render(clean, seed, frame)
    fr.splat()
    return fr.layers[0].clone()


class FrameData:
    """Device copies of one training / evaluation sample: two consecutive
    frames (clean radiance and G-buffer) and the motion of the second.
    reference() gives the HDR target of either frame: the clean image (the
    exact expectation of the renderer stand-in) or the 64-spp mean of the
    stand-in, rendered once per sample and kept."""

    def __init__(self, pair: dict, seed: int = 0):
        c = lambda a: torch.from_numpy(a).contiguous().cuda()
        self.clean_prev, self.clean = c(pair["clean_prev"]), c(pair["clean"])
        self.gprev = {k: c(v) for k, v in pair["gbuf_prev"].items()}
        self.g = {k: c(v) for k, v in pair["gbuf"].items()}
        self.mv = c(pair["mv"])
        self.H, self.W = self.clean.shape[1:]
        self.seed = seed
        self._ref64 = {}

    def reference(self, kind: str = "clean", prev: bool = False) -> torch.Tensor:
        if kind == "clean":
            return self.clean_prev if prev else self.clean
        if kind != "spp64":
            raise ValueError(f"unknown reference {kind}")
        if prev not in self._ref64:
            self._ref64[prev] = render_reference(self.clean_prev if prev else self.clean,
                                                 seed=0x64000000 + self.seed, frame=int(not prev))
        return self._ref64[prev]


ESTIMATORS = {"relaxed": B.SPP_ESTIMATOR_RELAXED,
              "straight_through": B.SPP_ESTIMATOR_STRAIGHT_THROUGH,
              "gumbel": B.SPP_ESTIMATOR_GUMBEL,
              "dasr": B.SPP_ESTIMATOR_DASR}
GUMBEL_LAMBDA = 10.0  # inverse temperature of the Gumbel-softmax relaxation


class Renderer:
    """Per-frame sampling / reconstruction state for B frames of W x H.

    estimator selects the gradient of the discretisation (Sec. 4.3, and the
    ablation of Sec. 7): "relaxed" (the ramp), "straight_through" (hard
    forward), "gumbel" (relaxed forward that traces every extra sample) or
    "dasr" (deterministic rounding with the surrogate gradient of Sec. 4.1,
    whose reference radiance is the clean image).  With train=False the
    straight-through and Gumbel models run the hard test-time rule; DASR
    keeps its deterministic rounding."""

    def __init__(self, B_: int, W: int, H: int, budget: float, dither_mask=None,
                 estimator: str = "relaxed", train: bool = True):
        if estimator not in ESTIMATORS:
            raise ValueError(f"unknown estimator {estimator}")
        self.B, self.W, self.H, self.budget = B_, W, H, budget
        self.estimator, self.train = estimator, train
        # blue-noise rank mask (device int16 [T][T]) or None for white noise
        self.dither = dither_mask
        # the Gumbel forward traces the extra sample of every pixel; rounding
        # to the nearest integer adds at most half a sample per pixel
        cap_budget = (budget + 1.0 if (estimator == "gumbel" and train)
                      else budget + 0.5 if estimator == "dasr" else budget)
        self.frames = [Frame(W, H, LEVELS, max_budget=cap_budget) for _ in range(B_)]
        self.cur_clean = [None] * B_
        self.cur_seed = [0] * B_
        self.tm = B.make_tonemap()
        self.hdr_prev = [_zeros(3, H, W) for _ in range(B_)]
        self.warped = [_zeros(3, H, W) for _ in range(B_)]
        self.prev_ldr = [_zeros(3, H, W) for _ in range(B_)]
        self.ref = [_zeros(3, H, W) for _ in range(B_)]
        self.mask = _zeros(H, W, dtype=torch.uint8)
        self.hats = [[_zeros(3, H >> l, W >> l) for l in range(LEVELS)] for _ in range(B_)]
        self.hdr = [_zeros(3, H, W) for _ in range(B_)]
        self.ldr = [_zeros(3, H, W) for _ in range(B_)]
        self.loss = [_zeros(4)[:1] for _ in range(B_)]
        self.g_ldr = _zeros(3, H, W)
        self.g_hdr = [_zeros(3, H >> l, W >> l) for l in range(LEVELS)]
        self.g_noisy = [_zeros(3, H >> l, W >> l) for l in range(LEVELS)]
        self.g_warped = _zeros(3, H, W)
        self.g_s = _zeros(W * H)
        self.mse = torch.zeros(2, dtype=torch.float64, device="cuda")[:1]
        self.dws = Predictor._aligned(B.spp_density_backward_workspace_bytes())
        self.cur_params = [None] * B_
        # temporal term of the objective: previous tone-mapped output and
        # reference, warped to the current frame
        self.ldr_prev = [_zeros(3, H, W) for _ in range(B_)]
        self.wldr_prev = [_zeros(3, H, W) for _ in range(B_)]
        self.wref_prev = [_zeros(3, H, W) for _ in range(B_)]
        self.tmp = _zeros(3, H, W)

    def _alloc(self, fr, d, params):
        if self.dither is not None:
            fr.alloc_dithered(d, params, self.dither)
        else:
            fr.alloc(d, params)

    def params(self, frame: int, seed: int):
        dasr = self.estimator == "dasr"
        gumbel = self.estimator == "gumbel" and self.train
        hard = self.estimator != "relaxed" and not gumbel and not dasr
        return B.make_params(self.budget, uniform_fraction=PHI, seed=seed, frame=frame, hard=hard,
                             gumbel=gumbel, dasr=dasr, lam=GUMBEL_LAMBDA if gumbel else 10.0)

    def previous_frame(self, b: int, d, logits, clean, seed: int, frame: int):
        """Frame t-1 of sample b (no temporal term); its output goes to hdr_prev[b]."""
        fr = self.frames[b]
        self._alloc(fr, d, self.params(frame, seed))
        fr.render(clean, seed ^ 0xC0FFEE, frame)
        fr.splat()
        out = fr.reconstruct(logits, tm=self.tm)
        self.hdr_prev[b].copy_(out)
        self.ldr_prev[b].copy_(fr.ldr)

    def warp_previous(self, b: int, mv):
        B.check(B.spp_warp_previous(self.hdr_prev[b], mv, self.W, self.H, self.warped[b]), "warp")
        B.check(B.spp_tonemap_image(self.warped[b], self.W, self.H, self.tm, self.prev_ldr[b]),
                "tonemap")

    def current_frame(self, b: int, d, logits, clean, seed: int, frame: int):
        """Frame t of sample b, level by level (the coarse outputs are kept
        for the backward), with the temporal term over warped[b]."""
        fr = self.frames[b]
        self.cur_params[b] = self.params(frame, seed)
        self.cur_clean[b], self.cur_seed[b] = clean, seed ^ 0xC0FFEE
        self._alloc(fr, d, self.cur_params[b])
        fr.render(clean, seed ^ 0xC0FFEE, frame)
        fr.splat()
        hats = self.hats[b]
        for l in range(LEVELS - 1, 0, -1):
            B.check(B.spp_reconstruct_level(fr.layers[l], logits[l], logits[l].shape[0],
                                            hats[l + 1] if l + 1 < LEVELS else None, None, None,
                                            self.W >> l, self.H >> l, None, hats[l], None),
                    "level")
        B.check(B.spp_reconstruct_level(fr.layers[0], logits[0], logits[0].shape[0], hats[1],
                                        self.warped[b], self.mask, self.W, self.H, self.tm,
                                        self.hdr[b], self.ldr[b]), "level 0")

    def reference(self, b: int, hdr_ref):
        """The tone-mapped target of sample b from its HDR reference."""
        B.check(B.spp_tonemap_image(hdr_ref, self.W, self.H, self.tm, self.ref[b]), "tonemap")

    def temporal_references(self, b: int, hdr_ref_prev, mv):
        """W(I_{t-1}) and W(I_ref,{t-1}) of Eq. loss_temporal: the previous
        tone-mapped output and reference warped to frame t."""
        B.check(B.spp_warp_previous(self.ldr_prev[b], mv, self.W, self.H, self.wldr_prev[b]),
                "warp")
        B.check(B.spp_tonemap_image(hdr_ref_prev, self.W, self.H, self.tm, self.tmp), "tonemap")
        B.check(B.spp_warp_previous(self.tmp, mv, self.W, self.H, self.wref_prev[b]), "warp")

    def backward(self, b: int, d, logits, g_logits, objective: str = "l1"):
        """Loss of sample b and its gradient into g_logits (level 0 planes
        0..53 and the density plane 54, levels 1 and 2).  objective "l1" is
        Eq. loss_spatial with m = 1; "combined" is Eq. loss_combined (needs
        temporal_references first)."""
        fr = self.frames[b]
        n = 3 * self.W * self.H
        if objective == "combined":
            B.check(B.spp_combined_loss(self.ldr[b], self.ref[b], self.wldr_prev[b],
                                        self.wref_prev[b], n, 1.25, 1.0, self.loss[b], self.g_ldr),
                    "combined loss")
        else:
            B.check(B.spp_l1_loss(self.ldr[b], self.ref[b], n, self.loss[b], self.g_ldr), "l1")
        g = self.g_hdr[0]
        g.zero_()
        B.check(B.spp_tonemap_backward(self.hdr[b], self.W, self.H, self.tm, self.g_ldr, g),
                "tonemap backward")
        for t in self.g_noisy:
            t.zero_()
        self.g_warped.zero_()
        hats = self.hats[b]
        for l in range(LEVELS):
            gc = self.g_hdr[l + 1] if l + 1 < LEVELS else None
            if gc is not None:
                gc.zero_()
            B.check(B.spp_reconstruct_level_backward(
                fr.layers[l], logits[l], logits[l].shape[0], hats[l + 1] if l + 1 < LEVELS else None,
                self.warped[b] if l == 0 else None, self.mask if l == 0 else None,
                self.W >> l, self.H >> l, self.g_hdr[l], g_logits[l], self.g_noisy[l], gc,
                self.g_warped if l == 0 else None), "level backward")
        B.check(B.spp_pyramid_backward(self.g_noisy, self.W, self.H, LEVELS, self.g_noisy[0]),
                "pyramid backward")
        B.check(B.spp_splat_backward_estimator(
            fr.offsets, fr.counts, fr.rgb, fr.s, fr.layers[0], self.g_noisy[0], fr.holdout_w,
            fr.capacity, self.W, self.H, self.cur_params[b], ESTIMATORS[self.estimator],
            self.cur_clean[b], self.cur_seed[b], self.g_s), "splat backward")
        B.check(B.spp_density_backward(d, self.W * self.H, self.budget, PHI, self.g_s,
                                       g_logits[3], self.dws), "density backward")

    def psnr(self, b: int) -> float:
        B.check(B.spp_mse(self.ldr[b], self.ref[b], 3 * self.W * self.H, self.mse), "mse")
        m = float(self.mse.item())
        return -10.0 * math.log10(max(m, 1e-30))


def random_tonemap(rng) -> "B.spp_tonemap":
    """A tone map of the training family (Sec. 5): contrast and saturation in
    [0.8, 1.2], exposure in [-1, 1], shadow and highlight in [0.2, 0.9]."""
    return B.make_tonemap(alpha=float(rng.uniform(0.8, 1.2)), beta=float(rng.uniform(0.8, 1.2)),
                          exposure=float(rng.uniform(-1.0, 1.0)),
                          shadow=float(rng.uniform(0.2, 0.9)),
                          highlight=float(rng.uniform(0.2, 0.9)))


class Trainer:
    """Trains the predictor on batches of two-frame samples.

    objective "l1" (Eq. loss_spatial, m = 1) or "combined" (Eq.
    loss_combined with the temporal term); random_tmo draws a tone map of
    the training family per step; total_steps enables cosine annealing of
    the learning rate; betas and weight_decay are AdamW's (the paper uses
    (0.8, 0.985) and 0.02); reference "clean" (the exact expectation of the
    renderer stand-in) or "spp64" (its 64-spp mean) is the target of the
    loss."""

    def __init__(self, theta: torch.Tensor, batch: int, size: int, budget: float = 0.25,
                 lr: float = 1e-3, weight_decay: float = 1e-4, objective: str = "l1",
                 betas=(0.9, 0.999), random_tmo: bool = False, total_steps: int | None = None,
                 seed: int = 0, dither_mask=None, estimator: str = "relaxed",
                 reference: str = "clean"):
        import numpy as np
        if reference not in ("clean", "spp64"):
            raise ValueError(f"unknown reference {reference}")
        self.reference = reference
        self.net = Predictor(theta, batch, size, size, train=True)
        self.rnd = Renderer(batch, size, size, budget, dither_mask, estimator=estimator)
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

    def step(self, samples: list[FrameData], seed: int) -> float:
        """One optimisation step on len(samples) == batch samples; returns
        the mean loss (reading it synchronises)."""
        net, rnd = self.net, self.rnd
        f_prev, f_cur = 2 * self.step_index, 2 * self.step_index + 1
        if self.random_tmo:
            rnd.tm = random_tonemap(self.rng)
        for b, s in enumerate(samples):
            net.features(b, s.gprev["albedo"], s.gprev["normal"], s.gprev["depth"], s.mv, None)
        net.forward()
        for b, s in enumerate(samples):
            rnd.previous_frame(b, net.density[b], net.frame_logits(b, False), s.clean_prev,
                               seed + b, f_prev)
            rnd.warp_previous(b, s.mv)
            net.features(b, s.g["albedo"], s.g["normal"], s.g["depth"], s.mv, rnd.prev_ldr[b])
        net.forward()
        for b, s in enumerate(samples):
            logits = net.frame_logits(b, True)
            rnd.current_frame(b, net.density[b], logits, s.clean, seed + b, f_cur)
            rnd.reference(b, s.reference(self.reference))
            if self.objective == "combined":
                rnd.temporal_references(b, s.reference(self.reference, prev=True), s.mv)
            gl = [net.g_logits[0][b, :54], net.g_logits[1][b], net.g_logits[2][b],
                  net.g_logits[0][b, 54]]
            rnd.backward(b, net.density[b], logits, gl, self.objective)
        net.backward()
        net.adamw(self.current_lr(), self.wd, grad_scale=1.0 / len(samples), betas=self.betas)
        self.step_index += 1
        return float(sum(l.item() for l in rnd.loss)) / len(samples)


def evaluate(samples: list[FrameData], budget: float, theta: torch.Tensor | None,
             fixed_logits: list[torch.Tensor] | None = None, seed: int = 99,
             temporal: list | None = None, dither_mask=None,
             estimator: str = "relaxed", coverage: list | None = None) -> list[float]:
    """PSNR (tone-mapped sRGB against the tone-mapped clean image) of frame
    t of each sample.  theta None runs the plain method: uniform density
    d = 1 and the fixed logits (54 / 29 / 25 channels).  If ``temporal`` is
    a list, the temporal error mean |dI - dI_ref| of Eq. loss_temporal of
    each sample is appended to it; if ``coverage`` is a list, the frame's
    samples per pixel and its fraction of pixels without a sample are."""
    W, H = samples[0].W, samples[0].H
    rnd = Renderer(1, W, H, budget, dither_mask, estimator=estimator, train=False)
    net = Predictor(theta, 1, W, H) if theta is not None else None
    ones = torch.ones(H, W, device="cuda")
    out = []
    for i, s in enumerate(samples):
        if net is not None:
            net.features(0, s.gprev["albedo"], s.gprev["normal"], s.gprev["depth"], s.mv, None)
            net.forward()
            d, lg = net.density[0], net.frame_logits(0, False)
        else:
            d, lg = ones, [fixed_logits[0][:29], fixed_logits[1], fixed_logits[2]]
        rnd.previous_frame(0, d, lg, s.clean_prev, seed + i, 0)
        rnd.warp_previous(0, s.mv)
        if net is not None:
            net.features(0, s.g["albedo"], s.g["normal"], s.g["depth"], s.mv, rnd.prev_ldr[0])
            net.forward()
            d, lg = net.density[0], net.frame_logits(0, True)
        else:
            lg = [fixed_logits[0], fixed_logits[1], fixed_logits[2]]
        rnd.current_frame(0, d, lg, s.clean, seed + i, 1)
        rnd.reference(0, s.clean)
        out.append(rnd.psnr(0))
        if coverage is not None:
            fr = rnd.frames[0]
            coverage.append((fr.sample_count() / (W * H),
                             float((fr.counts == 0).float().mean().item())))
        if temporal is not None:
            # mean |dI - dI_ref|: the combined loss with the spatial weight 0
            rnd.temporal_references(0, s.clean_prev, s.mv)
            B.check(B.spp_combined_loss(rnd.ldr[0], rnd.ref[0], rnd.wldr_prev[0],
                                        rnd.wref_prev[0], 3 * W * H, 1.0, 0.0, rnd.loss[0], None),
                    "temporal error")
            temporal.append(float(rnd.loss[0].item()))
    return out
