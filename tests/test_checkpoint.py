"""Checkpoint and resume of training, host logic (CPU): the state of a
trainer round-trips through a file, the tone-map generator continues its
sequence, the BF16 operands are re-packed, and mismatched checkpoints are
refused without touching the trainer.  Trainer stand-ins with CPU tensors
carry the attributes the real trainers have."""
import numpy as np
import pytest
import torch


@pytest.fixture(scope="module")
def ck():
    from conftest import build_spp_lib
    build_spp_lib()
    from paper_2602_08642_gb300 import checkpoint
    return checkpoint


class FakeNet:
    def __init__(self, net, n, seed):
        g = torch.Generator().manual_seed(seed)
        self.net = net
        self.theta = torch.randn(n, generator=g)
        self.m = torch.randn(n, generator=g)
        self.v = torch.rand(n, generator=g)
        self.step_count = seed
        self.packs = 0

    def pack(self):
        self.packs += 1


class Trainer:  # the name a checkpoint of learned.Trainer records
    def __init__(self, seed, step_index=0):
        self.net = FakeNet(0, 50, seed)
        self.lr, self.wd, self.betas = 1e-3, 1e-4, (0.9, 0.999)
        self.objective, self.total_steps, self.random_tmo = "combined", 100, True
        self.rng = np.random.default_rng(seed)
        self.step_index = step_index


class _Pair:
    def __init__(self, seed):
        self.sampler = FakeNet(1, 30, seed)
        self.denoiser = FakeNet(2, 40, seed + 1)


class TwoStageTrainer:
    def __init__(self, seed):
        self.p = _Pair(seed)
        self.lr, self.wd, self.betas = 1e-3, 1e-4, (0.9, 0.999)
        self.objective, self.total_steps, self.random_tmo = "l1", None, False
        self.rng = np.random.default_rng(seed)
        self.step_index = 0


def test_round_trip_and_generator_continues(ck, tmp_path):
    a = Trainer(seed=3, step_index=17)
    a.rng.random(5)  # the generator has moved on
    path = str(tmp_path / "a.pt")
    ck.save(path, a)
    expect_next = a.rng.random(4)
    b = Trainer(seed=9)
    ck.load(path, b)
    for k in ("theta", "m", "v"):
        assert torch.equal(getattr(b.net, k), getattr(a.net, k))
    assert b.net.step_count == 3 and b.step_index == 17 and b.net.packs == 1
    assert np.array_equal(b.rng.random(4), expect_next)


def test_two_stage_trainer_round_trip(ck, tmp_path):
    a, b = TwoStageTrainer(4), TwoStageTrainer(8)
    path = str(tmp_path / "t.pt")
    ck.save(path, a)
    ck.load(path, b)
    for na, nb in ((a.p.sampler, b.p.sampler), (a.p.denoiser, b.p.denoiser)):
        assert torch.equal(na.theta, nb.theta) and torch.equal(na.v, nb.v)
        assert nb.packs == 1


def test_mismatches_are_refused_untouched(ck, tmp_path):
    a = Trainer(seed=1)
    st = ck.state(a)
    b = Trainer(seed=2)
    before = b.net.theta.clone()
    with pytest.raises(ValueError):
        ck.load_state(TwoStageTrainer(2), st)            # another kind of trainer
    b.lr = 2e-3
    with pytest.raises(ValueError):
        ck.load_state(b, st)                              # other optimiser settings
    b.lr = a.lr
    b.net.net = 1
    with pytest.raises(ValueError):
        ck.load_state(b, st)                              # another network
    b.net.net = 0
    b.net.m = torch.zeros(49)
    with pytest.raises(ValueError):
        ck.load_state(b, st)                              # another parameter count
    bad = dict(st, format=99)
    with pytest.raises(ValueError):
        ck.load_state(Trainer(seed=2), bad)
    assert torch.equal(b.net.theta, before) and b.net.packs == 0 and b.step_index == 0


def test_interrupted_write_keeps_the_earlier_checkpoint(ck, tmp_path, monkeypatch):
    a = Trainer(seed=5, step_index=4)
    path = str(tmp_path / "c.pt")
    ck.save(path, a)

    def fail(*args, **kw):
        raise OSError("disk full")
    monkeypatch.setattr(ck.torch, "save", fail)
    a.step_index = 9
    with pytest.raises(OSError):
        ck.save(path, a)
    monkeypatch.undo()
    b = Trainer(seed=6)
    ck.load(path, b)
    assert b.step_index == 4
