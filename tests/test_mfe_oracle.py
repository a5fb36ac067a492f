"""Pins of the oracle's minimum free energy (Section "Minimization", Eq.
min-problem: the min-sum semiring over the partition-function recursions).

Checked against what the model fixes independently of the oracle: brute-force
minimisation over every codon sequence and structure (integer costs, exact
equality), the cost of the oracle's own minimiser re-evaluated by the
independent loop-decomposition evaluator, the bound between the ensemble
free energy and the minimum, and the closed form with pairing impossible.
"""
import math

import numpy as np
import pytest

import bruteforce as bf
import oracle
import synth

P0 = synth.nn_params(0)


@pytest.mark.parametrize("res,weighted", [([12], False), ([10, 15], False), ([0, 1, 2], False),
                                          ([5, 7, 2], True), ([1, 18, 3, 6], False), ([14, 0, 19, 7], True)])
def test_mfe_equals_bruteforce(res, weighted):
    m = len(res)
    rng = np.random.default_rng(100 + m)
    lw = rng.normal(0, 0.5, (m, 6)) if weighted else None
    pb = rng.normal(0, 0.2, (61, 61)) if weighted else None
    q, kc, cod, par = oracle.mfe(P0, res, lw, pb)
    assert q == bf.mfe_bruteforce(P0, res, lw, pb)
    assert kc == q / 2.0 ** 32
    # the returned minimiser is a valid configuration with exactly that cost
    assert bf.config_cost(P0, res, cod, par, lw, pb) == q


@pytest.mark.parametrize("m,seed", [(8, 0), (15, 3), (25, 9)])
def test_mfe_traceback_and_ensemble_bound(m, seed):
    """-kT ln Z <= MFE <= -kT ln Z + kT ln(number of configurations), and the
    minimiser's independently evaluated cost equals the MFE."""
    rng = np.random.default_rng(seed)
    res = rng.integers(0, 20, m)
    lw = rng.normal(0, 0.5, (m, 6))
    pb = rng.normal(0, 0.2, (61, 61))
    q, kc, cod, par = oracle.mfe(P0, res, lw, pb)
    assert bf.config_cost(P0, res, cod, par, lw, pb) == q
    kT = 1.98717e-3 * (P0[180] + 273.15)
    F = -kT * oracle.inside(P0, res, lw, pb)
    n = 3 * m
    ncodon = np.prod([len(bf.codons_for(int(r))) for r in res], dtype=np.float64)
    log_configs = math.log(ncodon) + n * math.log(3.0)  # Motzkin-type bound on structures
    assert F <= kc + 1e-9
    assert kc <= F + kT * log_configs + 1e-9


def test_mfe_without_pairs_is_cheapest_codon_path():
    """Lysine codons (AAA, AAG) cannot pair with each other: the minimum is
    the cheapest codon choice under the soft constraints alone, a shortest
    path over the codon chain (closed form by dynamic programming over
    residues)."""
    m = 12
    res = [synth.AMINO_ACIDS.index("K")] * m
    rng = np.random.default_rng(5)
    lw = rng.normal(0, 0.5, (m, 6))
    pb = rng.normal(0, 0.2, (61, 61))
    q, _, cod, par = oracle.mfe(P0, res, lw, pb)
    kT = 1.98717e-3 * (P0[180] + 273.15)
    cods = bf.codons_for(res[0])
    ids = [bf.SENSE_ID[c] for c in cods]
    best = [bf.qcost(-(kT * lw[0][s])) for s in range(len(cods))]
    for r in range(1, m):
        best = [min(best[a] + bf.qcost(-(kT * pb[ids[a]][ids[b]])) for a in range(len(cods)))
                + bf.qcost(-(kT * lw[r][b])) for b in range(len(cods))]
    assert q == min(best)
    assert (par == -1).all()
