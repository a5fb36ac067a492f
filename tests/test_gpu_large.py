"""The 1000-aa (3000 nt) soft-weighted protein: FP32 scaled inside and
outside against the FP64 GPU form and against properties that hold at any
size, and 10,000 exact samples.  (The oracle cross-check of this protein is
its 150-aa prefix, in the golden tests of test_gpu_parity.)"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)


@pytest.fixture(scope="module")
def large():
    import paper_2604_19718_b300 as cf
    res, lw, pb = synth.workload("p1000_weighted")
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    out = {}
    for prec in (1, 0):
        lz = f.inside(prec)
        P, cm, pg = f.outside()
        out[prec] = (lz, P, cm, pg)
    out["samples"] = f.sample(10_000, 2024)  # from the last inside pass (FP64)
    f.inside(1)
    out["samples32"] = f.sample(2_000, 2025)
    f.close()
    return res, out


def test_fp32_matches_fp64(large):
    res, out = large
    lz32, P32, cm32, _ = out[1]
    lz64, P64, cm64, _ = out[0]
    assert abs(lz32 - lz64) <= 1e-6 * abs(lz64)
    assert np.abs(cm32 - cm64).max() <= 1e-5
    assert np.abs(P32 - P64).max() <= 1e-5


def test_invariants(large):
    res, out = large
    for prec in (0, 1):
        lz, P, cm, pg = out[prec]
        assert np.isfinite(lz) and lz > 0
        assert np.abs(P - P.T).max() == 0
        assert P.min() >= -1e-6 and P.max() <= 1 + 1e-6
        assert np.abs(P.sum(1) - 1).max() <= 1e-4
        assert np.abs(cm.sum(1) - 1).max() <= (1e-9 if prec == 0 else 1e-5)
        for r, a in enumerate(res):
            assert np.all(cm[r, len(oracle.codons_of(a)):] == 0)


def _valid(res, cod, par):
    n = 3 * len(res)
    for c, p in zip(cod, par):
        for r, a in enumerate(res):
            assert c[r] in oracle.codons_of(a)
        stack = []
        for i in range(n):
            j = p[i]
            if j < 0:
                continue
            assert p[j] == i and abs(j - i) >= 4
            if j > i:
                stack.append(j)
            else:
                assert stack and stack.pop() == i  # pseudoknot-free


def test_samples(large):
    res, out = large
    cod, par = out["samples"]
    assert cod.shape == (10_000, 1000) and par.shape == (10_000, 3000)
    _valid(res, cod[:50], par[:50])
    _valid(res, out["samples32"][0][:20], out["samples32"][1][:20])
    cm = out[0][2]
    N = len(cod)
    worst = 0.0
    for r in range(0, 1000, 7):
        for s, cid in enumerate(oracle.codons_of(res[r])):
            p = min(max(cm[r, s], 0.0), 1.0)
            z = abs(np.mean(cod[:, r] == cid) - p) / (math.sqrt(p * (1 - p) / N) + 1e-12)
            worst = max(worst, z if p * (1 - p) * N > 1 else 0)
    assert worst < 5.0
