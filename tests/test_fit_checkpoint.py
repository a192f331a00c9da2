"""Checkpoint and resume of the transfer-function fit, on CPU tensors: a fit that
stops between checkpoints and is resumed from the last one ends bit for bit where
the uninterrupted fit ends (logits, Adam moments and loss history)."""

import numpy as np
import pytest
import torch

from paper_2605_19737_gb300.fit import adam_fit


class _Stop(Exception):
    pass


def _problem(seed=20260519):
    g = torch.Generator().manual_seed(seed)
    tf0 = torch.rand((1, 64, 4), generator=g, dtype=torch.float32)
    target = torch.rand((1, 64, 4), generator=g, dtype=torch.float32)
    w = torch.rand((1, 64, 4), generator=g, dtype=torch.float32)
    return tf0, lambda x: (w * (x - target) ** 2).mean()


def test_resume_reproduces_uninterrupted_fit(tmp_path):
    tf0, loss = _problem()
    ref_tf, ref_losses, _ = adam_fit(loss, tf0, steps=23, lr=5e-2)
    ck = str(tmp_path / "fit.pt")
    calls = {"n": 0}

    def crashing(x):
        calls["n"] += 1
        if calls["n"] == 13:  # dies inside step 13, after the checkpoint of step 10
            raise _Stop
        return loss(x)

    with pytest.raises(_Stop):
        adam_fit(crashing, tf0, steps=23, lr=5e-2, checkpoint=ck, every=5)
    st = torch.load(ck, weights_only=False)
    assert st["step"] == 10 and len(st["losses"]) == 10
    tf, losses, _ = adam_fit(loss, tf0, steps=23, lr=5e-2, checkpoint=ck, every=5)
    assert torch.equal(tf, ref_tf)
    np.testing.assert_array_equal(losses, ref_losses)
    assert torch.load(ck, weights_only=False)["step"] == 23
    # a finished checkpoint resumes to the same result without further steps
    tf2, losses2, _ = adam_fit(loss, tf0, steps=23, lr=5e-2, checkpoint=ck, every=5)
    assert torch.equal(tf2, ref_tf) and losses2 == losses


def test_fit_decreases_loss():
    tf0, loss = _problem(7)
    _, losses, ms = adam_fit(loss, tf0, steps=50, lr=5e-2)
    assert losses[-1] < 0.5 * losses[0] and ms >= 0.0
