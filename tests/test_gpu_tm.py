"""The paper's tensor-based free energy model on the GPU (cf_tm_inside)
against the oracle (oracle/tensor_model.py, pinned in tests/test_tm_oracle.py):

* log Z in both precisions for synthetic models of gamma 1-4 and 1-3 pair
  conformations, with and without the spectral-radius renormalisation, on
  proteins of 1-8 residues with codon weights and pair bonuses, and on a
  40-residue protein (120 nt: many staging steps of the cell kernel and a
  ragged last step);
* the renormalisation's radii equal the eigenvalue routine's;
* new codon weights on the same problem (cf_set_weights) give the oracle's
  value for them; a repeated call gives the same bits; the argument checks;
* at 450 nt (more cells per length than one wave of CTAs): repeated calls
  give the same bits in both precisions, binary32 agrees with binary64, and
  both layouts give the same binary64 log Z.
Tolerances: binary64 1e-11 relative (the recursion's sums in another
order); binary32 1e-6 relative to max(1, |log Z|) (the accuracy bar of the
nearest-neighbour path)."""
import numpy as np
import pytest

import synth
from oracle import tensor_model as tm

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)


def _cf():
    import paper_2604_19718_b300 as cf
    return cf


def _oracle(V, B, S, res, lw, pb, normalize):
    if normalize:
        V, B = tm.normalize(V, B)
    return tm.logz(V, B, S, res, lw, pb)


CASES = [(1, 1, [7], True), (2, 1, [3, 11], True), (3, 2, [0, 9, 2, 14], True), (4, 2, [5, 1, 18, 12, 3], True),
         (4, 3, list(range(1, 9)), True), (2, 2, [10, 15, 4, 6, 19, 8], False)]


@pytest.mark.parametrize("g,nrho,res,norm", CASES)
def test_logz_equals_oracle(g, nrho, res, norm):
    cf = _cf()
    V, B, S = synth.tm_params(10 * g + nrho, g, nrho)
    rng = np.random.default_rng(len(res))
    lw = rng.normal(0, 0.5, (len(res), 6))
    pb = rng.normal(0, 0.2, (61, 61))
    ref = _oracle(V, B, S, res, lw, pb, norm)
    model = cf.TensorModel(V, B, S, normalize=norm)
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    l64 = f.tm_inside(model, cf.CF_FP64)
    l32 = f.tm_inside(model, cf.CF_FP32_SCALED)
    assert f.tm_inside(model, cf.CF_FP32_SCALED) == l32  # deterministic
    f.close()
    model.close()
    assert abs(l64 - ref) <= 1e-11 * max(1.0, abs(ref))
    assert abs(l32 - ref) <= 1e-6 * max(1.0, abs(ref))


def test_40_residues_and_new_weights():
    cf = _cf()
    V, B, S = synth.tm_params(3, 4, 2)
    res = synth.residues_dirichlet(40, 7)
    rng = np.random.default_rng(9)
    lw = rng.normal(0, 0.5, (40, 6))
    pb = rng.normal(0, 0.2, (61, 61))
    model = cf.TensorModel(V, B, S)
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    ref = _oracle(V, B, S, res, lw, pb, True)
    l64 = f.tm_inside(model, cf.CF_FP64)
    l32 = f.tm_inside(model, cf.CF_FP32_SCALED)
    assert abs(l64 - ref) <= 1e-11 * abs(ref)
    assert abs(l32 - ref) <= 1e-6 * abs(ref)
    lw2 = rng.normal(0, 0.5, (40, 6))
    f.set_weights(lw2, pb)
    ref2 = _oracle(V, B, S, res, lw2, pb, True)
    assert abs(f.tm_inside(model, cf.CF_FP64) - ref2) <= 1e-11 * abs(ref2)
    f.close()
    model.close()


def test_450_nt_repeatable_and_layout_independent():
    """At 150 residues each length's launch has more cells than one wave of
    CTAs; the binary64 log Z repeats to the bit, binary32 agrees within the
    bar, and the single-codon layout gives the same binary64 log Z (exact
    arithmetic on the same sums, up to rounding order)."""
    cf = _cf()
    V, B, S = synth.tm_params(0, 4, 2)
    model = cf.TensorModel(V, B, S)
    res = synth.residues_dirichlet(150, 1)
    out = {}
    for layout in (0, 1):
        f = cf.CodonFold(P0)
        cf.cf_set_layout(f.prob, layout)
        f.set_protein(res)
        a = f.tm_inside(model, cf.CF_FP64)
        assert f.tm_inside(model, cf.CF_FP64) == a
        b = f.tm_inside(model, cf.CF_FP32_SCALED)
        assert f.tm_inside(model, cf.CF_FP32_SCALED) == b
        f.close()
        assert abs(a - b) <= 1e-6 * abs(a)
        out[layout] = a
    model.close()
    assert abs(out[0] - out[1]) <= 1e-11 * abs(out[0])


def test_radius_and_argument_checks():
    cf = _cf()
    V, B, S = synth.tm_params(5, 3, 2)
    model = cf.TensorModel(V, B, S)
    r = model.radius()
    for x in range(4):
        assert r[x] == pytest.approx(tm.spectral_radius(V[x]), rel=1e-11)
    f = cf.CodonFold(P0)
    with pytest.raises(cf.CFError) as e:
        f.tm_inside(model)  # no protein yet
    assert e.value.status == cf.CF_ESTATE
    f.set_protein([1, 2, 3])
    with pytest.raises(cf.CFError) as e:
        cf.cf_tm_inside(f.prob, model.h, 7)
    assert e.value.status == cf.CF_EINVAL
    f.close()
    model.close()
    with pytest.raises(cf.CFError) as e:
        cf.TensorModel(np.ones((4, 5, 5)), np.ones((1, 4, 4, 5, 5)), np.ones((5, 5)))  # gamma > 4
    assert e.value.status == cf.CF_EINVAL
    with pytest.raises(cf.CFError) as e:
        cf.TensorModel(np.zeros((4, 2, 2)), np.ones((1, 4, 4, 2, 2)), np.ones((2, 2)))  # radius 0
    assert e.value.status == cf.CF_EINVAL
