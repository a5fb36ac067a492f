"""GPU sampler (through the C ABI): exactness and reproducibility.

* the distribution of (codon sequence, structure) matches the exact
  probabilities enumerated by brute force (chi-square, 3 residues);
* codon and pair frequencies match the oracle's marginals within 4.5 sigma;
* a sample depends only on (seed, index): identical across calls and across
  batch sizes (different launch shapes), different across seeds;
* every sample is a valid member of the ensemble (encodes the protein,
  pseudoknot-free, canonical pairs, hairpins >= 3).
"""
import math

import numpy as np
import pytest

import bruteforce as bf
import oracle
import synth

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)


def _fold(res, lw=None, pb=None, prec=1):
    import paper_2604_19718_b300 as cf
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    f.inside(prec)
    return f


def _valid(res, cod, par):
    n = 3 * len(res)
    allowed = [set(oracle.codons_of(r)) for r in res]
    for c, x in zip(cod, par):
        assert all(int(c[r]) in allowed[r] for r in range(len(res)))
        seq = [bf._IDX[ch] for cid in c for ch in bf.SENSE[cid]]
        stack = []
        for i in range(n):
            j = x[i]
            if j < 0:
                continue
            assert x[j] == i and j != i
            if j > i:
                assert j - i >= 4 and (seq[i], seq[j]) in bf.PAIRS
                stack.append(j)
            else:
                assert stack and stack[-1] == i
                stack.pop()


@pytest.mark.parametrize("prec", [0, 1])
def test_exact_distribution(prec):
    res = [1, 9, 10]
    rng = np.random.default_rng(1)
    lw = rng.normal(0, 0.5, (3, 6))
    pb = rng.normal(0, 0.3, (61, 61))
    b = bf.summary(P0, res, lw, pb)
    probs = {}
    for _, cids, pt, w in b["ensemble"]:
        probs[(cids, pt)] = probs.get((cids, pt), 0.0) + w / b["Z"]
    f = _fold(res, lw, pb, prec)
    N = 200000
    cod, par = f.sample(N, 99)
    f.close()
    cnt = {}
    for c, x in zip(map(tuple, cod), map(tuple, par)):
        cnt[(c, x)] = cnt.get((c, x), 0) + 1
    assert all(k in probs for k in cnt), "sample outside the ensemble"
    chi, dof = 0.0, 0
    for k, pr in probs.items():
        e = N * pr
        if e >= 5:
            chi += (cnt.get(k, 0) - e) ** 2 / e
            dof += 1
    z = ((chi / dof) ** (1 / 3) - (1 - 2 / (9 * dof))) / math.sqrt(2 / (9 * dof))
    assert z < 3.8, (chi, dof)


def test_marginals_and_validity():
    res, lw, pb = synth.workload("p300_weighted")
    res, lw = res[:30], lw[:30]
    o = oracle.outside(P0, res, lw, pb)
    f = _fold(res, lw, pb, 1)
    N = 20000
    cod, par = f.sample(N, 5)
    f.close()
    _valid(res, cod[:500], par[:500])
    for r in range(len(res)):
        for s, cid in enumerate(oracle.codons_of(res[r])):
            p = o["codon"][r, s]
            fr = np.mean(cod[:, r] == cid)
            assert abs(fr - p) <= 4.5 * math.sqrt(p * (1 - p) / N) + 1e-9
    n = 3 * len(res)
    emp = np.zeros((n, n))
    rows = np.repeat(np.arange(n)[None, :], N, 0)
    cols = np.where(par < 0, rows, par)
    np.add.at(emp, (rows.ravel(), cols.ravel()), 1.0)
    emp /= N
    sd = np.sqrt(o["P"] * (1 - o["P"]) / N)
    assert np.all(np.abs(emp - o["P"]) <= 4.5 * sd + 2.0 / N)


def test_reproducible_per_seed_any_launch_shape():
    res, lw, pb = synth.workload("p300_weighted")
    res, lw = res[:60], lw[:60]
    f = _fold(res, lw, pb, 1)
    c1, p1 = f.sample(64, 1234)
    c2, p2 = f.sample(64, 1234)
    c3, p3 = f.sample(3000, 1234)  # more samples than resident warps: other launch shape
    c4, p4 = f.sample(64, 1235)
    f.close()
    assert np.array_equal(c1, c2) and np.array_equal(p1, p2)
    assert np.array_equal(c1, c3[:64]) and np.array_equal(p1, p3[:64])
    assert not (np.array_equal(c1, c4) and np.array_equal(p1, p4))
    _valid(res, c3[:200], p3[:200])


def test_full_size_samples_valid():
    res, lw, pb = synth.workload("p300_dirichlet")
    f = _fold(res, lw, pb, 1)
    cod, par = f.sample(1000, 7)
    f.close()
    _valid(res, cod[:100], par[:100])
    # codon frequencies against the full-size oracle marginals
    from pathlib import Path
    g = Path(__file__).resolve().parent / "golden" / "p300_dirichlet.npz"
    if g.exists():
        cm = np.load(g)["codon"]
        N = len(cod)
        for r in range(len(res)):
            for s, cid in enumerate(oracle.codons_of(res[r])):
                p = cm[r, s]
                assert abs(np.mean(cod[:, r] == cid) - p) <= 5.0 * math.sqrt(p * (1 - p) / N) + 1e-9
