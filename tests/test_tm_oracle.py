"""Pins of the tensor-model oracle (oracle/tensor_model.py) to values fixed by
the model's definition (paper SI "Tensor-based free energy models", Eq.
general-model; Eq. amino-q for the codon weights), independent of its own
recursion:
  * the recursion equals the brute-force sum over codon sequences, structures
    and rho assignments (1-3 residues, gamma 1-3, one or two rho);
  * a scalar model (gamma 1, V = S = 1, one pair weight b on each side of a
    pair) counts structures: Z = prod_r |C(psi_r)| * sum_p N_p b^(2p), with
    N_p the number of pseudoknot-free structures of p pairs (hairpins >= 3),
    counted by hand: 6 nt [1, 3], 9 nt [1, 15, 15, 1];
  * with no pair weights Z is the codon-weighted trace of the product of the
    unpaired matrices along the sequence, written out for one residue;
  * codon weights factor out: lw shifted by a constant c per residue adds
    m c to log Z;
  * the spectral-radius renormalisation (SI "Free energy model
    renormalization") leaves every V with spectral radius 1 (diagonal and
    2 x 2 closed forms) and scales B by 1/sqrt(r_x r_y);
  * the codon table has the standard genetic code's 61 sense codons with the
    per-amino-acid counts of the C oracle."""
import math

import numpy as np
import pytest

import oracle
from oracle import tensor_model as tm


def _model(rng, g, nrho):
    V = rng.uniform(0.2, 1.0, (4, g, g))
    B = rng.uniform(0.0, 1.5, (nrho, 4, 4, g, g))
    S = rng.uniform(0.1, 1.0, (g, g))
    return V, B, S


@pytest.mark.parametrize("g,nrho", [(1, 1), (2, 2), (3, 1)])
@pytest.mark.parametrize("res", [[3], [4, 7], [0, 9, 2], [12, 18, 5]])
def test_recursion_equals_brute_force(g, nrho, res):
    rng = np.random.default_rng(10 * g + nrho + len(res))
    V, B, S = _model(rng, g, nrho)
    lw = rng.normal(0, 0.5, (len(res), 6))
    pb = rng.normal(0, 0.3, (61, 61))
    a = tm.logz(V, B, S, res, lw, pb)
    b = tm.brute_force_logz(V, B, S, res, lw, pb)
    assert abs(a - b) <= 1e-12 * max(1.0, abs(b))


@pytest.mark.parametrize("res,counts", [([1, 9], [1, 3]), ([7, 0, 12], [1, 15, 15, 1])])
def test_scalar_model_counts_structures(res, counts):
    b = 1.7
    V = np.ones((4, 1, 1))
    B = np.full((1, 4, 4, 1, 1), b)
    S = np.ones((1, 1))
    ncod = math.prod(len(tm.codon_states(r)) for r in res)
    Z = ncod * sum(c * b ** (2 * p) for p, c in enumerate(counts))
    assert abs(tm.logz(V, B, S, res) - math.log(Z)) <= 1e-12
    assert abs(tm.brute_force_logz(V, B, S, res) - math.log(Z)) <= 1e-12


def test_no_pairs_is_the_trace_of_the_unpaired_product():
    rng = np.random.default_rng(3)
    V, _, S = _model(rng, 3, 1)
    B = np.zeros((1, 4, 4, 3, 3))
    lw = rng.normal(0, 0.5, (1, 6))
    aa = 1  # arginine: six codons
    Z = 0.0
    for slot, (_, b1, b2, b3) in enumerate(tm.codon_states(aa)):
        Z += math.exp(lw[0, slot]) * np.trace(S @ V[b1] @ V[b2] @ V[b3])
    assert abs(tm.logz(V, B, S, [aa], lw) - math.log(Z)) <= 1e-12


def test_codon_weight_shift_adds_to_logz():
    rng = np.random.default_rng(4)
    V, B, S = _model(rng, 2, 2)
    res = [5, 11, 16, 2]
    lw = rng.normal(0, 0.5, (4, 6))
    a = tm.logz(V, B, S, res, lw)
    b = tm.logz(V, B, S, res, lw + 0.25)
    assert abs((b - a) - 4 * 0.25) <= 1e-10


def test_spectral_normalisation():
    assert tm.spectral_radius(np.diag([0.5, 2.5, 1.0])) == pytest.approx(2.5, rel=1e-14)
    a, b, c, d = 1.0, 2.0, 3.0, 4.0  # eigenvalues (a + d)/2 +- sqrt(((a - d)/2)^2 + bc)
    lam = (a + d) / 2 + math.sqrt(((a - d) / 2) ** 2 + b * c)
    assert tm.spectral_radius([[a, b], [c, d]]) == pytest.approx(lam, rel=1e-13)
    rng = np.random.default_rng(5)
    V, B, _ = _model(rng, 3, 2)
    Vn, Bn = tm.normalize(V, B)
    r = [tm.spectral_radius(V[x]) for x in range(4)]
    for x in range(4):
        assert tm.spectral_radius(Vn[x]) == pytest.approx(1.0, rel=1e-12)
        for y in range(4):
            assert np.allclose(Bn[:, x, y] * math.sqrt(r[x] * r[y]), B[:, x, y], rtol=1e-14, atol=0)


def test_codon_table():
    total = 0
    for aa in range(20):
        st = tm.codon_states(aa)
        assert len(st) == len(oracle.codons_of(aa))
        total += len(st)
    assert total == 61
    assert [len(tm.codon_states(a)) for a in (1, 10, 15, 12, 17)] == [6, 6, 6, 1, 1]  # R, L, S, M, W
