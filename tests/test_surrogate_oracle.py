"""Pins of the surrogate reference (oracle/surrogate.py): its hand-written
forward and backward against PyTorch's float64 conv1d and autograd, an
independent library path on the same definition."""
import numpy as np
import torch
import torch.nn.functional as F

import synth
from oracle import surrogate as sg


def _torch_loss(flat, windows, G):
    p = [torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in sg.unpack(flat)]
    loss = 0.0
    for bases, Gw in zip(windows, G):
        n = len(bases)
        h = F.one_hot(torch.tensor(np.asarray(bases, dtype=np.int64)), 4).T.to(torch.float64)[None]
        for l in range(4):
            h = F.relu(F.conv1d(h, p[2 * l], p[2 * l + 1], padding=2))
        g = (p[8][None, :, None] * h).sum() / n + p[9][0]
        loss = loss + (g - Gw / n) ** 2 / len(windows)
    loss.backward()
    return float(loss), np.concatenate([a.grad.numpy().ravel() for a in p])


def test_shapes_agree():
    assert [tuple(s) for s in sg.SHAPES] == synth.SURROGATE_SHAPES
    assert sg.NPARAM == len(synth.surrogate_init(0)) == 63041


def test_forward_backward_equal_torch_autograd():
    rng = np.random.default_rng(4)
    flat = synth.surrogate_init(1)
    flat[np.r_[1280:1344]] = rng.normal(0, 0.1, 64)  # non-zero biases
    windows = [rng.integers(0, 4, n) for n in (7, 30, 61)]
    G = rng.normal(-40, 10, 3)
    l1, g1 = sg.loss_and_grad(flat, windows, G)
    l2, g2 = _torch_loss(flat, windows, G)
    assert abs(l1 - l2) < 1e-12 * max(1, abs(l2))
    assert np.abs(g1 - g2).max() < 1e-10 * max(1.0, np.abs(g2).max())
    pred = sg.predict(flat, windows)
    for b, pv in zip(windows, pred):
        g, _ = sg.forward_one(flat, b)
        assert abs(pv - len(b) * g) < 1e-12


def test_gradient_central_differences():
    rng = np.random.default_rng(5)
    flat = synth.surrogate_init(2)
    windows = [rng.integers(0, 4, n) for n in (12, 9)]
    G = np.array([-5.0, -3.0])
    _, g = sg.loss_and_grad(flat, windows, G)
    h = 1e-6
    for i in rng.choice(len(flat), 12, replace=False):
        e = np.zeros_like(flat)
        e[i] = h
        fd = (sg.loss_and_grad(flat + e, windows, G)[0] - sg.loss_and_grad(flat - e, windows, G)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(g[i])), i
