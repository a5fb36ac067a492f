"""Checkpointed interior-loop partial sums (the adjoint's largest
intermediate): the inside pass keeps two diagonals and every 64th diagonal,
the outside pass recomputes each 64-diagonal block from its checkpoint, and
the sampler evaluates the partial sums from their definition.

* checkpointed and stored forms give the same log Z (bit for bit) and the
  same outside outputs (the recomputation repeats the inside's operation
  order; only the outside's atomic scatters vary run to run), both
  precisions;
* the checkpointed sampler draws from the exact distribution (chi-square
  against brute force at 3 residues) and matches the oracle's codon
  marginals;
* the 3000-nt workload is checkpointed by default and matches the oracle on
  its 150-residue prefix; a 4500-nt protein completes in both precisions and
  they agree to the accuracy bar.
"""
import math
from pathlib import Path

import numpy as np
import pytest

import bruteforce as bf
import oracle
import synth

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)
GOLD = Path(__file__).resolve().parent / "golden"


def _cf():
    import paper_2604_19718_b300 as cf
    return cf


def _run(res, lw, pb, prec, ck):
    cf = _cf()
    f = cf.CodonFold(P0)
    cf.cf_set_checkpoint(f.prob, ck)
    f.set_protein(res, lw, pb)
    lz = f.inside(prec)
    P, cm, pg = f.outside()
    assert cf.cf_checkpointed(f.prob) == bool(ck)
    return f, lz, P, cm, pg


@pytest.mark.parametrize("prec", [1, 0])
def test_checkpointed_equals_stored(prec):
    res, lw, pb = synth.workload("p300_weighted")  # 900 nt: 14 blocks of 64 diagonals
    f0, lz0, P0_, cm0, pg0 = _run(res, lw, pb, prec, 0)
    f1, lz1, P1, cm1, pg1 = _run(res, lw, pb, prec, 1)
    f0.close()
    f1.close()
    assert lz1 == lz0
    # the binary32 outside's atomic scatters vary run to run at this level
    # (the stored form against itself spreads the same way)
    assert np.abs(P1 - P0_).max() <= 1e-6
    assert np.abs(cm1 - cm0).max() <= 1e-6
    assert np.abs(pg1 - pg0).max() <= 1e-5
    g = np.load(GOLD / "p300_weighted.npz")
    assert np.abs(P1 - g["P"]).max() <= (1e-5 if prec == 1 else 2e-7)


@pytest.mark.parametrize("prec", [1, 0])
def test_checkpointed_sampler_exact_distribution(prec):
    cf = _cf()
    res = [1, 9, 10]
    rng = np.random.default_rng(1)
    lw = rng.normal(0, 0.5, (3, 6))
    pb = rng.normal(0, 0.3, (61, 61))
    b = bf.summary(P0, res, lw, pb)
    probs = {}
    for _, cids, pt, w in b["ensemble"]:
        probs[(cids, pt)] = probs.get((cids, pt), 0.0) + w / b["Z"]
    f = cf.CodonFold(P0)
    cf.cf_set_checkpoint(f.prob, 1)
    f.set_protein(res, lw, pb)
    f.inside(prec)
    N = 200000
    cod, par = f.sample(N, 77)
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


def test_checkpointed_sampler_marginals():
    cf = _cf()
    res, lw, pb = synth.workload("p300_weighted")
    res, lw = res[:40], lw[:40]
    o = oracle.outside(P0, res, lw, pb)
    f = cf.CodonFold(P0)
    cf.cf_set_checkpoint(f.prob, 1)
    f.set_protein(res, lw, pb)
    f.inside(1)
    N = 20000
    cod, par = f.sample(N, 5)
    f.close()
    for r in range(len(res)):
        for s, cid in enumerate(oracle.codons_of(res[r])):
            p = o["codon"][r, s]
            assert abs(np.mean(cod[:, r] == cid) - p) <= 4.5 * math.sqrt(p * (1 - p) / N) + 1e-9
    n = 3 * len(res)
    emp = np.zeros((n, n))
    rows = np.repeat(np.arange(n)[None, :], N, 0)
    cols = np.where(par < 0, rows, par)
    np.add.at(emp, (rows.ravel(), cols.ravel()), 1.0)
    emp /= N
    sd = np.sqrt(o["P"] * (1 - o["P"]) / N)
    assert np.all(np.abs(emp - o["P"]) <= 4.5 * sd + 2.0 / N)


def test_3000_nt_checkpointed_by_default_and_prefix_golden():
    cf = _cf()
    res, lw, pb = synth.workload("p1000_weighted")
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    lz = f.inside(cf.CF_FP32_SCALED)
    _, cm, _ = f.outside(False, True, False)
    assert cf.cf_checkpointed(f.prob)
    cod, par = f.sample(256, 3)
    f.close()
    assert np.isfinite(lz) and np.abs(cm.sum(1) - 1).max() <= 1e-5
    assert (cod >= 0).all()
    g = np.load(GOLD / "p1000_weighted_prefix150.npz")
    h = cf.CodonFold(P0)
    cf.cf_set_checkpoint(h.prob, 1)
    h.set_protein(res[:150], lw[:150])
    lz2 = h.inside(cf.CF_FP32_SCALED)
    P2, cm2, _ = h.outside()
    h.close()
    assert abs(lz2 - float(g["logZ"])) <= 1e-6 * abs(float(g["logZ"]))
    assert np.abs(P2 - g["P"]).max() <= 1e-5 and np.abs(cm2 - g["codon"]).max() <= 1e-5


def test_4500_nt_both_precisions_agree():
    """1500 residues (4500 nt, Dirichlet(1) composition, seed 4 continued,
    codon weights ~ N(0, 0.5)): checkpointed binary32 against checkpointed
    binary64 at the accuracy bar."""
    cf = _cf()
    rng = np.random.default_rng(44)
    freqs = rng.dirichlet(np.ones(20))
    res = rng.choice(20, 1500, p=freqs)
    lw = rng.normal(0.0, 0.5, (1500, 6))
    f = cf.CodonFold(P0)
    f.set_protein(res, lw)
    lz32 = f.inside(cf.CF_FP32_SCALED)
    P32, cm32, _ = f.outside(True, True, False)
    lz64 = f.inside(cf.CF_FP64)
    P64, cm64, _ = f.outside(True, True, False)
    assert cf.cf_checkpointed(f.prob)
    f.close()
    assert abs(lz32 - lz64) <= 1e-6 * abs(lz64)
    assert np.abs(P32 - P64).max() <= 1e-5
    assert np.abs(cm32 - cm64).max() <= 1e-5
