"""Host logic of the autograd wrapper and the weight ascent, run on the CPU
against an oracle-backed stand-in for the GPU problem.

The stand-in answers set_weights / inside / outside with the oracle, so these
tests check LogZ's forward/backward plumbing (argument order, masks, the
stale-forward guard) and the ascent loop, and they pin the oracle's adjoint
once more against central finite differences of its own log Z.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2604_19718_b300 import adjoint

P0 = synth.nn_params(0)


class OracleFold:
    """CodonFold's weight/inside/outside surface, computed by the oracle."""

    def __init__(self, residues):
        self.res = np.asarray(residues)
        self.m = len(self.res)
        self.n = 3 * self.m
        self.lw = self.pb = None

    def set_weights(self, lw=None, pb=None):
        self.lw, self.pb = lw, pb
        return self

    def inside(self, precision=0):
        return oracle.inside(P0, self.res, self.lw, self.pb)

    def outside(self, pair_prob=True, codon=True, pair_grad=True):
        o = oracle.outside(P0, self.res, self.lw, self.pb)
        if codon is not False:
            codon[...] = torch.as_tensor(o["codon"])
        if pair_grad is not False:
            pair_grad[...] = torch.as_tensor(o["pair_grad"])
        return None, codon, pair_grad


def _protein(m, seed):
    res = synth.residues_uniform(m, seed)
    lw, pb = synth.soft_weights(m, seed + 7)
    return res, lw, pb


def test_codon_counts_match_genetic_code():
    for k, a in enumerate("ARNDCQEGHILKMFPSTWYV"):
        assert adjoint.CODONS_PER_AA[a] == len(oracle.codons_of(k))
    assert sum(adjoint.CODONS_PER_AA.values()) == 61


def test_frequency_targets_are_distributions_on_valid_slots():
    res = synth.residues_uniform(30, 5)
    aa = synth.to_string(res)
    f = adjoint.frequency_targets(aa, synth.ascent_targets(30))
    mask = adjoint.slot_mask(aa)
    assert np.allclose(f.sum(axis=1), 1.0) and np.all(f[~mask] == 0) and np.all(f[mask] > 0)


@pytest.mark.parametrize("seed", [1, 2])
def test_autograd_gradients_equal_central_differences(seed):
    res, lw, pb = _protein(3, seed)
    fold = OracleFold(res)
    lw_t = torch.tensor(lw, requires_grad=True)
    pb_t = torch.tensor(pb, requires_grad=True)
    z = adjoint.LogZ.apply(lw_t, pb_t, fold, 0)
    z.backward()
    mask = adjoint.slot_mask(synth.to_string(res))
    h = 1e-4

    def f(lw_, pb_):
        return oracle.inside(P0, res, lw_, pb_)
    for r in range(3):
        for s in range(6):
            e = np.zeros_like(lw)
            e[r, s] = h
            fd = (f(lw + e, pb) - f(lw - e, pb)) / (2 * h)
            assert abs(fd - float(lw_t.grad[r, s])) < 1e-7, (r, s)
            if not mask[r, s]:
                assert float(lw_t.grad[r, s]) == 0.0
    g = pb_t.grad.numpy()
    used = np.argwhere(g > 1e-3)[:6]
    assert len(used) >= 1
    for c1, c2 in list(used) + [(0, 1)]:
        e = np.zeros_like(pb)
        e[c1, c2] = h
        fd = (f(lw, pb + e) - f(lw, pb - e)) / (2 * h)
        assert abs(fd - g[c1, c2]) < 1e-7, (c1, c2)


def test_stale_forward_is_rejected():
    res, lw, pb = _protein(2, 3)
    fold = OracleFold(res)
    a = torch.tensor(lw, requires_grad=True)
    z1 = adjoint.LogZ.apply(a, None, fold, 0)
    adjoint.LogZ.apply(a.detach(), None, fold, 0)
    with pytest.raises(RuntimeError, match="evaluated again"):
        z1.backward()


def test_weight_ascent_reaches_targets():
    res = synth.residues_uniform(4, 11)
    aa = synth.to_string(res)
    fstar = adjoint.frequency_targets(aa, synth.ascent_targets(4))
    fold = OracleFold(res)
    lw, hist = adjoint.weight_ascent(fold, aa, fstar, steps=40, lr=1.0)
    obj = [h["objective"] for h in hist]
    assert all(b >= a - 1e-12 for a, b in zip(obj, obj[1:]))  # concave, step 1 <= 1/curvature
    gaps = [h["max_gap"] for h in hist]
    assert gaps[-1] < 0.03 * gaps[0]  # plain gradient ascent: slow along low-curvature slots
    p = oracle.outside(P0, res, lw.numpy())["codon"]
    mask = adjoint.slot_mask(aa)
    assert np.abs(p - fstar)[mask].max() < gaps[-1]
