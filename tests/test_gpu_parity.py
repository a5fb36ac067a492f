"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Element-by-element comparison on the same seeded inputs: log Z, the full pair
probability matrix, codon marginals and codon-pair gradients, in both the
binary64 form and the binary32 form with per-diagonal power-of-two scaling.
Tolerances: binary64 1e-9 (relative for log Z, absolute for marginals) and
2e-7 for pair probabilities, which the ABI returns as binary32; binary32 1e-6
relative for log Z and 1e-5 absolute for probabilities (the accuracy bar of
the workload).
Full-size workloads are compared against values the oracle wrote with
tests/golden/make_golden.py.
"""
import math
from pathlib import Path

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

P0 = synth.nn_params(0)
GOLD = Path(__file__).resolve().parent / "golden"
TOL = {0: (1e-9, 1e-9, 2e-7), 1: (1e-6, 1e-5, 1e-5)}  # precision -> (logZ rel, marginal abs, P abs)


def _cf():
    import paper_2604_19718_b300 as cf
    return cf


def _gpu(res, lw, pb, prec):
    cf = _cf()
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    lz = f.inside(prec)
    P, cm, pg = f.outside()
    f.close()
    return lz, P, cm, pg


def _check(o, g, prec, res):
    lz, P, cm, pg = g
    tl, tp, tP = TOL[prec]
    assert abs(lz - o["logZ"]) <= tl * max(1.0, abs(o["logZ"])), (lz, o["logZ"])
    assert np.abs(P - o["P"]).max() <= tP
    assert np.abs(cm - o["codon"]).max() <= tp
    assert np.abs(pg - o["pair_grad"]).max() <= tp * max(1, len(res) // 10)


CASES = {
    "one_residue": ([12], False),
    "two": ([10, 15], False),
    "three": ([0, 1, 2], False),
    "four_weighted": ([5, 7, 2, 14], True),
    "p8_uniform": (list(synth.workload("p8_uniform")[0]), False),
    "p21_weighted": (list(np.random.default_rng(21).integers(0, 20, 21)), True),
    "p47_weighted": (list(np.random.default_rng(47).integers(0, 20, 47)), True),
}


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_vs_oracle(name, prec):
    res, wts = CASES[name]
    m = len(res)
    rng = np.random.default_rng(m)
    lw = rng.normal(0, 0.5, (m, 6)) if wts else None
    pb = rng.normal(0, 0.2, (61, 61)) if wts else None
    o = oracle.outside(P0, res, lw, pb)
    _check(o, _gpu(res, lw, pb, prec), prec, res)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["p300_dirichlet", "p300_weighted", "p1000_weighted_prefix150"])
def test_full_size_golden(name, prec):
    path = GOLD / f"{name}.npz"
    if not path.exists():
        pytest.skip(f"golden {name} not generated")
    g = np.load(path)
    if name.startswith("p1000"):
        res, lw, _ = synth.workload("p1000_weighted")
        res, lw, pb = res[:150], lw[:150], None
    else:
        res, lw, pb = synth.workload(name)
    lz, P, cm, pg = _gpu(res, lw, pb, prec)
    tl, tp, tP = TOL[prec]
    assert abs(lz - float(g["logZ"])) <= tl * abs(float(g["logZ"]))
    assert np.abs(cm - g["codon"]).max() <= tp
    # every element of the pair-probability matrix (at 900 nt the outside
    # chain runs its 256-thread cells on diagonals with more than 296 cells)
    assert g["P"].shape == P.shape
    assert np.abs(P - g["P"]).max() <= tP
    assert np.abs(np.diag(P) - g["unpaired"]).max() <= tP
    assert np.abs(pg - g["pair_grad"]).max() <= 10 * tp


def test_invariants_fp32_full():
    res, lw, pb = synth.workload("p300_weighted")
    lz, P, cm, pg = _gpu(res, lw, pb, 1)
    assert np.abs(P - P.T).max() == 0
    assert P.min() >= -1e-5 and P.max() <= 1 + 1e-5
    assert np.abs(P.sum(1) - 1).max() <= 1e-4
    assert np.abs(cm.sum(1) - 1).max() <= 1e-5
    assert abs(pg.sum() - (len(res) - 1)) <= 1e-3


def test_errors():
    cf = _cf()
    f = cf.CodonFold(P0)
    with pytest.raises(cf.CFError) as e:
        f.inside()
    assert e.value.status == cf.CF_ESTATE
    with pytest.raises(cf.CFError) as e:
        f.set_protein("MAXW")
    assert e.value.status == cf.CF_EINVAL
    with pytest.raises(cf.CFError) as e:
        f.set_protein("MAW", np.full((3, 6), np.nan))
    assert e.value.status == cf.CF_EINVAL
    f.set_protein("MAW")
    with pytest.raises(cf.CFError) as e:
        f.outside()
    assert e.value.status == cf.CF_ESTATE
    f.close()


def test_repeatable_and_device_outputs():
    import torch
    cf = _cf()
    res, lw, pb = synth.workload("p300_weighted")
    res, lw = res[:40], lw[:40]
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    a = f.inside(1)
    b = f.inside(1)
    assert a == b
    n = f.n
    Pd = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    cmd = torch.zeros((len(res), 6), dtype=torch.float64, device="cuda")
    bmd = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
    cf.cf_outside(f.prob, Pd, cmd, base_marg=bmd)
    torch.cuda.synchronize()
    P, cm, _, bm = f.outside(base=True)
    # binary32: the adjoint scatters and the transfer-gradient sums use atomics,
    # whose order varies between runs (measured spread 1e-9 at this size)
    assert np.array_equal(Pd.cpu().numpy(), P) or np.abs(Pd.cpu().numpy() - P).max() < 1e-6
    assert np.abs(cmd.cpu().numpy() - cm).max() < 1e-7
    assert np.abs(bmd.cpu().numpy() - bm).max() < 1e-7
    f.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_same_length_protein_reuses_tables(prec):
    """A second protein of the same length on the same problem (tables and
    graphs reused) gives what a fresh problem gives, and matches the oracle."""
    cf = _cf()
    res, lw, pb = synth.workload("p300_weighted")
    a, b = slice(0, 40), slice(40, 80)
    f = cf.CodonFold(P0)
    f.set_protein(res[a], lw[a], pb)
    f.inside(prec)
    f.outside()
    f.sample(64, 5)
    f.set_protein(res[b], lw[b], pb)
    lz = f.inside(prec)
    P, cm, pg = f.outside()
    cod, par = f.sample(64, 5)
    f.close()
    g = cf.CodonFold(P0)
    g.set_protein(res[b], lw[b], pb)
    lz2 = g.inside(prec)
    P2, cm2, pg2 = g.outside()
    cod2, par2 = g.sample(64, 5)
    g.close()
    assert lz == lz2
    assert np.abs(P - P2).max() < 1e-6 and np.abs(cm - cm2).max() < 1e-9
    assert np.array_equal(cod, cod2) and np.array_equal(par, par2)
    o = oracle.outside(P0, res[b], lw[b], pb)
    tl, tm, tp = TOL[prec]
    assert abs(lz - o["logZ"]) <= tl * max(1.0, abs(o["logZ"]))
    assert np.abs(cm - o["codon"]).max() <= tm and np.abs(P - o["P"]).max() <= tp


@pytest.mark.parametrize("prec", [0, 1])
def test_base_marginals_vs_oracle(prec):
    """Per-base marginals p_i(b) (Eq. marginal-base) against the oracle's, and
    each position's four sum to one."""
    cf = _cf()
    res, wts = CASES["p47_weighted"]
    m = len(res)
    rng = np.random.default_rng(m)
    lw = rng.normal(0, 0.5, (m, 6))
    pb = rng.normal(0, 0.2, (61, 61))
    o = oracle.outside(P0, res, lw, pb)
    want = oracle.base_marginals(res, o["codon"])
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    f.inside(prec)
    _, _, _, bm = f.outside(base=True)
    f.close()
    assert bm.shape == (3 * m, 4)
    assert np.abs(bm - want).max() <= TOL[prec][1]
    assert np.abs(bm.sum(axis=1) - 1.0).max() <= TOL[prec][1]
