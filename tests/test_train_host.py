"""Host logic of the training driver (no GPU): the cosine schedule, the draws
of media and inputs, the checkpoint calls, and resumption at a step, checked
with a stand-in network that records what it is asked to do."""
import math

import pytest

np = pytest.importorskip("numpy")

from paper_2604_23265_gb300 import train


class Recorder:
    def __init__(self):
        self.calls = []

    def train_step(self, ctx, batch, lr):
        self.calls.append((ctx, tuple(batch), lr))
        return 1.0 / (1 + len(self.calls))


def _setup():
    ctxs = ["m0", "m1", "m2"]
    inputs = [[f"{c}:{k}" for k in range(6)] for c in ctxs]
    return ctxs, inputs


def test_schedule_and_draws():
    ctxs, inputs = _setup()
    r = Recorder()
    losses = train.train(r, ctxs, inputs, steps=10, batch=4, lr0=2e-3, seed=3)
    assert len(losses) == 10 and len(r.calls) == 10
    for it, (ctx, batch, lr) in enumerate(r.calls):
        assert lr == pytest.approx(0.5 * 2e-3 * (1 + math.cos(math.pi * it / 10)))
        assert len(set(batch)) == 4 and all(b.startswith(ctx + ":") for b in batch)


def test_resume_replays_the_draws_and_continues_the_schedule():
    ctxs, inputs = _setup()
    full = Recorder()
    train.train(full, ctxs, inputs, steps=12, batch=3, lr0=1e-3, seed=5)
    resumed = Recorder()
    train.train(resumed, ctxs, inputs, steps=12, batch=3, lr0=1e-3, seed=5, start_step=7)
    assert resumed.calls == full.calls[7:]


def test_checkpoints_every_k_steps_and_at_the_end():
    ctxs, inputs = _setup()
    seen = []
    train.train(Recorder(), ctxs, inputs, steps=9, batch=2, seed=1,
                checkpoint=lambda it, net, ls: seen.append((it, len(ls))), every=4)
    assert seen == [(0, 0), (4, 4), (8, 8), (9, 9)]
