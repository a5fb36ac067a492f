"""The surrogate's own CUDA forward/backward against the float64 reference
(oracle/surrogate.py), its optimiser, and what the trained network gains
when it pre-screens candidates for the exact window DP."""
import numpy as np
import pytest

import synth
from oracle import surrogate as sg

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)


def bf16_round(x):
    """Round float64 values to the nearest bfloat16 (ties to even)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _params(seed):
    rng = np.random.default_rng(seed)
    p = synth.surrogate_init(seed)
    off = 0
    for s in synth.SURROGATE_SHAPES:
        k = int(np.prod(s))
        if len(s) == 3:
            p[off:off + k] = bf16_round(p[off:off + k])
        else:
            p[off:off + k] = rng.normal(0, 0.05, k)
        off += k
    return p.astype(np.float32).astype(np.float64)


def _windows(lens, seed):
    rng = np.random.default_rng(seed)
    ws = [rng.integers(0, 4, n).astype(np.uint8) for n in lens]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    return ws, np.concatenate(ws), off


def test_forward_and_gradient_equal_reference():
    import paper_2604_19718_b300 as cf
    p = _params(3)
    lens = [5, 17, 64, 131, 200, 256]
    ws, b, off = _windows(lens, 4)
    G = np.random.default_rng(5).normal(-60, 20, len(lens))
    sur = cf.Surrogate(p, max_batch=8)
    loss, g = sur.grad(b, off, G)
    lr, gr = sg.loss_and_grad(p, ws, G)
    assert abs(loss - lr) <= 1e-4 * abs(lr)
    scale = np.abs(gr).max()
    assert np.abs(g - gr).max() <= 1e-3 * scale
    # per block too, so that a small layer cannot hide behind a large one
    o = 0
    for s in synth.SURROGATE_SHAPES:
        k = int(np.prod(s))
        blk = gr[o:o + k]
        assert np.abs(g[o:o + k] - blk).max() <= 1e-3 * max(np.abs(blk).max(), 1e-6 * scale), s
        o += k
    pred = sur.predict(b, off)
    ref = sg.predict(p, ws)
    assert np.abs(pred - ref).max() <= 1e-4 * np.abs(ref).max()
    sur.close()


def test_predict_chunks_devices_and_edge_windows():
    import torch

    import paper_2604_19718_b300 as cf
    p = _params(6)
    lens = [0, 1, 3, 40, 256, 90, 12, 7, 255, 33, 64]
    ws, b, off = _windows(lens, 7)
    small = cf.Surrogate(p, max_batch=3)
    big = cf.Surrogate(p, max_batch=64)
    a = small.predict(b, off)
    c = big.predict(b, off)
    assert np.array_equal(a, c)
    assert a[0] == 0.0  # an empty window predicts n g = 0
    d = torch.zeros(len(lens), dtype=torch.float32, device="cuda")
    cf.cf_surrogate_predict(big.h, torch.tensor(b, device="cuda"), torch.tensor(off, device="cuda"), d)
    assert np.array_equal(d.cpu().numpy(), c)
    ref = sg.predict(p, [w for w in ws if len(w)])
    assert np.abs(c[1:] - ref).max() <= 1e-4 * np.abs(ref).max()
    with pytest.raises(cf.CFError) as e:
        big.predict(np.zeros(300, np.uint8), np.array([0, 300]))
    assert e.value.status == cf.CF_EINVAL
    with pytest.raises(cf.CFError):
        small.grad(b, off, np.zeros(len(lens)))  # batch above max_batch
    small.close()
    big.close()


def test_adam_step_matches_reference_update():
    import paper_2604_19718_b300 as cf
    p = _params(8)
    ws, b, off = _windows([50, 80, 120], 9)
    G = np.array([-30.0, -50.0, -70.0])
    sur = cf.Surrogate(p, max_batch=4)
    _, g = sur.grad(b, off, G)
    sur.train_step(b, off, G, 1e-3)
    q = sur.params()
    # first Adam step: m/(1-b1) = g, v/(1-b2) = g^2, so dp = -lr g / (|g| + eps)
    expect = p.astype(np.float32) - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.abs(q - expect).max() < 1e-6
    sur.close()


def _trained(n_train=60000, epochs=6):
    import paper_2604_19718_b300 as cf
    from paper_2604_19718_b300 import screen
    exact = screen.Windows(P0)
    res, slots, bases, off = synth.windows(n_train + 2000, seed=3)
    G = exact.free_energy(bases, off)
    tr = np.arange(n_train)
    b_tr, o_tr = screen.gather(bases, off, tr)
    sur = cf.Surrogate(synth.surrogate_init(0), max_batch=256)
    hist = screen.train(sur, b_tr, o_tr, G[tr], epochs=epochs, batch=256, lr=1e-3)
    return sur, exact, (res, slots, bases, off, G), hist


def test_training_and_prescreen_gain():
    from paper_2604_19718_b300 import screen
    sur, exact, (res, slots, bases, off, G), hist = _trained()
    assert hist[-1] < 0.5 * hist[0]
    held = np.arange(len(res) - 2000, len(res))
    b_h, o_h = screen.gather(bases, off, held)
    pred = sur.predict(b_h, o_h)
    n = np.diff(o_h)
    base = n * np.mean(G[:-2000] / np.diff(off)[:-2000])  # length-only predictor
    mse_s = np.mean((pred - G[held]) ** 2)
    mse_b = np.mean((base - G[held]) ** 2)
    assert mse_s < 0.5 * mse_b, (mse_s, mse_b)
    # design: 1024 uniform candidates per window; surrogate picks 32 for the
    # exact DP, against 32 random candidates scored exactly
    rng = np.random.default_rng(11)
    gain = []
    for w in held[:8]:
        cands = screen.uniform_candidates(res[w], 1024, rng)
        s = screen.prescreen(sur, exact, res[w], cands, top=32)
        d = screen.dp_only(exact, res[w], cands[:32])
        gain.append(d["best_G"] - s["best_G"])
    assert np.mean(gain) > 0, gain
    sur.close()
    exact.close()


def test_tensor_core_prediction_matches_cuda_cores_and_reference():
    """Prediction on the 5th-generation tensor cores (tcgen05 MMA, 128-row
    tiles straddling windows, BF16 hi/lo activations) against the CUDA-core
    path with FP32 activations and against the float64 reference, on windows
    of every length class (empty, shorter than a tap span, one tile, several
    tiles) in batches that split across chunks."""
    import paper_2604_19718_b300 as cf
    p = _params(11)
    rng = np.random.default_rng(12)
    lens = [0, 1, 2, 4, 5, 127, 128, 129, 256, 255] + list(rng.integers(60, 241, 300))
    ws, b, off = _windows(lens, 13)
    sur = cf.Surrogate(p, max_batch=128)
    cf.cf_surrogate_set_path(sur.h, 0)
    cc = sur.predict(b, off)
    cf.cf_surrogate_set_path(sur.h, 1)
    tc = sur.predict(b, off)
    tc2 = sur.predict(b, off)
    sur.close()
    nz = [i for i, w in enumerate(ws) if len(w) > 0]
    ref = sg.predict(p, [ws[i] for i in nz])
    scale = np.maximum(1.0, np.abs(cc))
    assert np.array_equal(tc, tc2)  # deterministic
    assert (np.abs(tc - cc) / scale).max() <= 1e-4
    assert np.abs(tc[nz] - ref).max() <= 1e-4 * np.abs(ref).max()
    assert tc[0] == 0.0 and cc[0] == 0.0
