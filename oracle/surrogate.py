"""Surrogate network reference -- TEST INFRASTRUCTURE ONLY.

Plain float64 NumPy forward and backward of the window free-energy surrogate
(a learned stand-in for the exact window partition function; the paper has
none, it only scores windows exactly).  Only ``tests/`` and ``bench.py``'s CPU
baseline may use it; the CUDA kernels share nothing with it.

Network, per window of n bases (A, C, G, U = 0..3):

* h0[c][t] = 1 if base t is c else 0, for t in [0, n), four channels;
* layer l = 1..4: pre_l[o][t] = b_l[o] + sum_{c, k} W_l[o][c][k] h_{l-1}[c][t + k - 2]
  (K = 5 taps, h_{l-1} read as zero outside [0, n)), h_l = max(pre_l, 0),
  64 output channels;
* g = (1/n) sum_{t, c} wh[c] h4[c][t] + bh, the predicted free energy per
  base; the predicted window free energy is n g (kcal/mol).

Training loss over a batch of B windows: (1/B) sum_w (g_w - G_w / n_w)^2.

Flat parameter order: W1 (64x4x5), b1, W2 (64x64x5), b2, W3, b3, W4, b4,
wh (64), bh (1).
"""
from __future__ import annotations

import numpy as np

C = 64      # channels
K = 5       # taps
HALF = K // 2
CIN = (4, 64, 64, 64)
SHAPES = []
for _cin in CIN:
    SHAPES += [(C, _cin, K), (C,)]
SHAPES += [(C,), (1,)]
NPARAM = int(sum(np.prod(s) for s in SHAPES))


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    out, o = [], 0
    for s in SHAPES:
        k = int(np.prod(s))
        out.append(flat[o:o + k].reshape(s))
        o += k
    return out


def _conv(W, b, h):
    """pre[o][t] = b[o] + sum_{c,k} W[o][c][k] h[c][t+k-HALF], zero padding."""
    cin, n = h.shape
    hp = np.zeros((cin, n + 2 * HALF))
    hp[:, HALF:HALF + n] = h
    pre = np.repeat(b[:, None], n, axis=1).astype(np.float64)
    for k in range(K):
        pre += W[:, :, k] @ hp[:, k:k + n]
    return pre


def forward_one(flat, bases):
    """Returns g (per-base prediction) and the activations h0..h4."""
    p = unpack(flat)
    n = len(bases)
    h = np.zeros((4, n))
    h[np.asarray(bases, dtype=np.int64), np.arange(n)] = 1.0
    hs = [h]
    for l in range(4):
        h = np.maximum(_conv(p[2 * l], p[2 * l + 1], h), 0.0)
        hs.append(h)
    g = float((p[8][:, None] * h).sum() / n + p[9][0])
    return g, hs


def predict(flat, windows):
    """Predicted window free energies n * g (kcal/mol)."""
    return np.array([len(b) * forward_one(flat, b)[0] for b in windows])


def loss_and_grad(flat, windows, G):
    """Batch loss and its gradient with respect to the flat parameters."""
    p = unpack(flat)
    grads = [np.zeros(s) for s in SHAPES]
    B = len(windows)
    loss = 0.0
    for bases, Gw in zip(windows, G):
        n = len(bases)
        g, hs = forward_one(flat, bases)
        r = g - Gw / n
        loss += r * r / B
        dg = 2.0 * r / B
        grads[9][0] += dg
        grads[8] += dg * hs[4].sum(axis=1) / n
        dh = np.repeat((dg * p[8] / n)[:, None], n, axis=1)
        for l in range(3, -1, -1):
            dpre = dh * (hs[l + 1] > 0)
            W = p[2 * l]
            grads[2 * l + 1] += dpre.sum(axis=1)
            hp = np.zeros((W.shape[1], n + 2 * HALF))
            hp[:, HALF:HALF + n] = hs[l]
            for k in range(K):
                grads[2 * l][:, :, k] += dpre @ hp[:, k:k + n].T
            if l > 0:
                # dh_{l-1}[c][s] = sum_{o,k} W[o][c][k] dpre[o][s-k+HALF]
                dp = np.zeros((C, n + 2 * HALF))
                dp[:, HALF:HALF + n] = dpre
                dh = np.zeros((W.shape[1], n))
                for k in range(K):
                    dh += W[:, :, k].T @ dp[:, K - 1 - k:K - 1 - k + n]
    return loss, np.concatenate([g.ravel() for g in grads])

