"""Checkpoint and resume of training.

A checkpoint holds what a trainer (learned.Trainer or
two_stage.TwoStageTrainer) needs to continue where it stopped:
- per network, the FP32 master parameters, AdamW's two moments and its step
  count (the BF16 operand image is re-packed from the parameters on load);
- the trainer's step index, which drives the cosine learning-rate schedule
  and the frame indices of the seeded sample streams;
- the state of the generator that draws the random tone maps;
- the optimiser settings, checked on load so that a run does not resume
  under different ones by mistake.

The sampling seeds of a step are arguments of the step itself, so the caller
resumes its own seed sequence.  The reconstruction backward accumulates with
FP32 atomics, so a resumed run follows the original closely but not bit for
bit.
"""
from __future__ import annotations

import os

import torch

FORMAT = 1
_SETTINGS = ("lr", "wd", "betas", "objective", "total_steps", "random_tmo")


def _networks(trainer) -> list:
    if hasattr(trainer, "net"):
        return [trainer.net]
    return [trainer.p.sampler, trainer.p.denoiser]


def _net_state(net) -> dict:
    host = lambda t: t.detach().to("cpu", torch.float32).clone()  # noqa: E731
    return {"net": int(net.net), "theta": host(net.theta), "m": host(net.m), "v": host(net.v),
            "adam_step": int(net.step_count)}


def state(trainer) -> dict:
    """Host copy of the trainer's state (tensors on the CPU)."""
    return {
        "format": FORMAT,
        "kind": type(trainer).__name__,
        "step_index": int(trainer.step_index),
        "rng": trainer.rng.bit_generator.state,
        "settings": {k: (list(getattr(trainer, k)) if k == "betas" else getattr(trainer, k))
                     for k in _SETTINGS},
        "nets": [_net_state(n) for n in _networks(trainer)],
    }


def load_state(trainer, st: dict) -> None:
    """Restores a state taken by state() into a trainer built with the same
    networks and settings; raises ValueError on any mismatch (nothing is
    changed then)."""
    if st.get("format") != FORMAT:
        raise ValueError(f"checkpoint format {st.get('format')!r}, expected {FORMAT}")
    if st.get("kind") != type(trainer).__name__:
        raise ValueError(f"checkpoint of a {st.get('kind')}, not a {type(trainer).__name__}")
    nets = _networks(trainer)
    if len(st["nets"]) != len(nets):
        raise ValueError("checkpoint holds a different number of networks")
    for net, ns in zip(nets, st["nets"]):
        if ns["net"] != int(net.net):
            raise ValueError(f"checkpoint network {ns['net']}, trainer network {int(net.net)}")
        for k in ("theta", "m", "v"):
            if ns[k].numel() != getattr(net, k).numel():
                raise ValueError(f"checkpoint {k} has {ns[k].numel()} values, "
                                 f"the network {getattr(net, k).numel()}")
    settings = {k: (list(getattr(trainer, k)) if k == "betas" else getattr(trainer, k))
                for k in _SETTINGS}
    if settings != st["settings"]:
        raise ValueError(f"optimiser settings differ: checkpoint {st['settings']}, "
                         f"trainer {settings}")
    for net, ns in zip(nets, st["nets"]):
        net.theta.copy_(ns["theta"])
        net.m.copy_(ns["m"])
        net.v.copy_(ns["v"])
        net.step_count = ns["adam_step"]
        net.pack()
    trainer.step_index = st["step_index"]
    trainer.rng.bit_generator.state = st["rng"]


def save(path: str, trainer) -> None:
    """Writes the trainer's state to path (through a temporary file in the
    same directory, renamed into place, so that an interrupted write leaves
    any earlier checkpoint intact)."""
    tmp = f"{path}.tmp{os.getpid()}"
    torch.save(state(trainer), tmp)
    os.replace(tmp, path)


def load(path: str, trainer) -> None:
    """Restores the state saved at path into the trainer (see load_state)."""
    load_state(trainer, torch.load(path, map_location="cpu", weights_only=True))
