"""Frequency matching through the library's inside/outside passes: the
binary64 iterates equal those driven by the oracle's marginals, and the
binary32 form converges on the 300-residue protein."""
import numpy as np
import pytest

import oracle
import synth

P0 = synth.nn_params(0)


@pytest.mark.gpu
def test_gpu_iterates_match_the_oracle():
    import paper_2604_19718_b300 as cf
    from paper_2604_19718_b300 import frequency as fq
    res = synth.residues_uniform(10, 4)
    aa = synth.to_string(res)
    fstar = np.exp(np.random.default_rng(104).normal(0.0, 1.0, 61))
    f = cf.CodonFold(P0)
    f.set_protein(res)
    xg, hg = fq.match_frequencies(fq.fold_marginals(f, precision=cf.CF_FP64), aa, fstar, rtol=1e-6)
    f.close()
    xo, ho = fq.match_frequencies(lambda lw: oracle.outside(P0, res, lw)["codon"], aa, fstar, rtol=1e-6)
    assert len(hg) == len(ho)
    assert np.allclose(hg, ho, rtol=1e-6, atol=1e-9)
    assert np.abs(xg - xo).max() < 1e-6


@pytest.mark.gpu
def test_gpu_fp32_converges_on_300_residues():
    import paper_2604_19718_b300 as cf
    from paper_2604_19718_b300 import frequency as fq
    res, _, _ = synth.workload("p300_dirichlet")
    aa = synth.to_string(res)
    fstar = np.exp(np.random.default_rng(3).normal(0.0, 1.0, 61))
    f = cf.CodonFold(P0)
    f.set_protein(res)
    x, hist = fq.match_frequencies(fq.fold_marginals(f), aa, fstar, rtol=0.002)
    b = fq.codon_counts(aa, fq.fold_marginals(f)(fq.slot_weights(aa, x)))
    f.close()
    bs = fq.target_counts(aa, fstar)
    act = bs > 0
    assert hist[-1] < 0.002 and len(hist) <= 30
    assert np.abs(np.log(b[act] / bs[act])).max() < 0.002
