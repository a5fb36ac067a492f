"""Frequency matching (Algorithm "Naive iterative algorithm for frequency
matching", with Anderson mixing) driven by the oracle's codon marginals on
small proteins: the result is the fixed point the algorithm defines (the
achieved codon counts equal the targets), and the table of codon slots agrees
with the oracle's codon lists."""
import numpy as np
import pytest

import oracle
import synth

P0 = synth.nn_params(0)


def _fq():
    from paper_2604_19718_b300 import frequency
    return frequency


def _case(m, seed):
    res = synth.residues_uniform(m, seed)
    aa = synth.to_string(res)
    fstar = np.exp(np.random.default_rng(seed + 100).normal(0.0, 1.0, 61))
    return res, aa, fstar


def _oracle_marginals(res):
    return lambda lw: oracle.outside(P0, res, lw)["codon"]


def test_slot_codon_ids_are_the_oracles_codon_lists():
    fq = _fq()
    aa = synth.AMINO_ACIDS
    ids = fq.slot_codon_ids(aa)
    for a in range(20):
        assert [int(c) for c in ids[a] if c >= 0] == oracle.codons_of(a)


def test_target_counts():
    fq = _fq()
    res, aa, fstar = _case(12, 1)
    b = fq.target_counts(aa, fstar)
    assert abs(b.sum() - len(aa)) < 1e-12
    # uniform bonuses: each residue spreads one count evenly over its codons
    u = fq.target_counts(aa, np.ones(61))
    ids = fq.slot_codon_ids(aa)
    want = np.zeros(61)
    for r in range(len(aa)):
        row = ids[r][ids[r] >= 0]
        want[row] += 1.0 / row.size
    assert np.abs(u - want).max() < 1e-15


@pytest.mark.parametrize("m,seed", [(6, 2), (10, 3)])
def test_converges_to_the_fixed_point(m, seed):
    fq = _fq()
    res, aa, fstar = _case(m, seed)
    x, hist = fq.match_frequencies(_oracle_marginals(res), aa, fstar, rtol=1e-6, depth=5)
    assert hist[-1] < 1e-6
    # the achieved counts at the returned bonuses equal the targets
    b = fq.codon_counts(aa, oracle.outside(P0, res, fq.slot_weights(aa, x))["codon"])
    bs = fq.target_counts(aa, fstar)
    act = bs > 0
    assert np.abs(np.log(b[act] / bs[act])).max() < 1e-6


def test_anderson_needs_fewer_evaluations_than_the_naive_iteration():
    fq = _fq()
    res, aa, fstar = _case(10, 4)
    _, naive = fq.match_frequencies(_oracle_marginals(res), aa, fstar, rtol=1e-6, depth=0, max_iter=400)
    _, anders = fq.match_frequencies(_oracle_marginals(res), aa, fstar, rtol=1e-6, depth=5)
    assert naive[-1] < 1e-6 and anders[-1] < 1e-6
    assert len(anders) < len(naive)
