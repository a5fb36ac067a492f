"""Batched fixed-sequence windows (cf_window_logz) against the oracle with
every residue clamped to one codon, against brute-force enumeration for
sequences of any length, and on the error paths."""
import math

import numpy as np
import pytest

import bruteforce as bf
import oracle
import synth

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)


def _prob():
    import paper_2604_19718_b300 as cf
    m = cf.cf_load_model(P0)
    return cf, m, cf.cf_problem_create(m, 0, 0)


def _clamped(res, slots):
    lw = np.full((len(res), 6), -np.inf)
    lw[np.arange(len(res)), slots] = 0.0
    return lw


def _run(cf, prob, bases, offsets):
    out = np.zeros(len(offsets) - 1)
    cf.cf_window_logz(prob, np.ascontiguousarray(bases, dtype=np.uint8),
                      np.ascontiguousarray(offsets, dtype=np.int64), out)
    return out


def test_windows_equal_clamped_oracle():
    cf, model, prob = _prob()
    res, slots, bases, off = synth.windows(64, seed=3)
    pick = list(range(10))
    # plus truncations to short and ragged whole-codon lengths
    cuts = [(10, 1), (11, 2), (12, 4), (13, 7), (14, 11), (15, 21)]
    seqs, ref = [], []
    for w in pick:
        seqs.append(bases[off[w]:off[w + 1]])
        ref.append(oracle.inside(P0, res[w], _clamped(res[w], slots[w])))
    for w, k in cuts:
        seqs.append(bases[off[w]:off[w] + 3 * k])
        ref.append(oracle.inside(P0, res[w][:k], _clamped(res[w][:k], slots[w][:k])))
    o2 = np.concatenate([[0], np.cumsum([len(s) for s in seqs])])
    got = _run(cf, prob, np.concatenate(seqs), o2)
    for g, r in zip(got, ref):
        assert abs(g - r) <= 1e-6 * max(1.0, abs(r)), (g, r)
    cf.cf_problem_free(prob)
    cf.cf_model_free(model)


def test_windows_equal_brute_force_any_length():
    cf, model, prob = _prob()
    p = bf.Params(P0)
    rng = np.random.default_rng(21)
    seqs, ref = [], []
    for n in (1, 4, 5, 9, 13, 14, 16):
        s = rng.integers(0, 4, n)
        z = 0.0
        for pt in bf.structures(list(s)):
            e = bf.energy(p, list(s), pt)
            if e is not None:
                z += math.exp(-e / p.kT)
        seqs.append(s)
        ref.append(math.log(z))
    o2 = np.concatenate([[0], np.cumsum([len(s) for s in seqs])])
    got = _run(cf, prob, np.concatenate(seqs), o2)
    assert np.abs(got - np.array(ref)).max() < 1e-5
    assert got[0] == 0.0 and got[1] == 0.0  # no pair fits in fewer than 5 bases
    cf.cf_problem_free(prob)
    cf.cf_model_free(model)


def test_device_and_host_buffers_and_repeat():
    import torch
    cf, model, prob = _prob()
    _, _, bases, off = synth.windows(300, seed=5)
    host = _run(cf, prob, bases, off)
    db = torch.tensor(bases, device="cuda")
    do = torch.tensor(off, device="cuda")
    dz = torch.zeros(len(off) - 1, dtype=torch.float64, device="cuda")
    cf.cf_window_logz(prob, db, do, dz)
    assert np.array_equal(dz.cpu().numpy(), host)
    assert np.array_equal(_run(cf, prob, bases, off), host)  # deterministic
    assert cf.cf_window_last_ms(prob) > 0
    cf.cf_problem_free(prob)
    cf.cf_model_free(model)


def test_window_errors():
    cf, model, prob = _prob()
    with pytest.raises(cf.CFError) as e:
        _run(cf, prob, np.array([0, 1, 5, 2, 3, 0], np.uint8), np.array([0, 6]))
    assert e.value.status == cf.CF_EINVAL
    with pytest.raises(cf.CFError) as e:
        _run(cf, prob, np.zeros(10, np.uint8), np.array([0, 6, 4]))
    assert e.value.status == cf.CF_EINVAL
    with pytest.raises(cf.CFError) as e:
        _run(cf, prob, np.zeros(1100, np.uint8), np.array([0, 1100]))
    assert e.value.status == cf.CF_EINVAL and "CF_WINDOW_MAX_N" in str(e.value)
    assert len(_run(cf, prob, np.zeros(0, np.uint8), np.array([0]))) == 0
    # the problem stays usable after an error
    assert _run(cf, prob, np.zeros(0, np.uint8), np.array([0, 0]))[0] == 0.0
    cf.cf_problem_free(prob)
    cf.cf_model_free(model)


def test_full_batch_sampled_against_oracle():
    """200,000 windows in one call; 12 sampled windows recomputed by the oracle."""
    cf, model, prob = _prob()
    res, slots, bases, off = synth.windows(200_000, seed=3)
    got = _run(cf, prob, bases, off)
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    rng = np.random.default_rng(9)
    for w in rng.choice(len(res), 12, replace=False):
        r = oracle.inside(P0, res[w], _clamped(res[w], slots[w]))
        assert abs(got[w] - r) <= 1e-6 * max(1.0, abs(r)), (w, got[w], r)
    cf.cf_problem_free(prob)
    cf.cf_model_free(model)
