"""The single-codon layout (cf_set_layout(prob, 1), paper Eq. single-tt): the
same protein gives the same log Z, pair probabilities, codon and base
marginals as the codon-state layout and the oracle, in both precisions, with
codon weights; the tensor-based model's log Z is the same in both layouts;
the state counts are the distinct first bases, (first, second) pairs and
third bases, 1.5-1.8 per position; the calls the layout does not serve are refused."""
import numpy as np
import pytest

import oracle
import synth
from oracle import tensor_model as tm

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)


def _cf():
    import paper_2604_19718_b300 as cf
    return cf


def _run(res, lw, layout, prec):
    cf = _cf()
    f = cf.CodonFold(P0)
    cf.cf_set_layout(f.prob, layout)
    f.set_protein(res, lw)
    lz = f.inside(prec)
    P, cm, _, bm = f.outside(True, True, False, base=True)
    lay, states = cf.cf_layout_states(f.prob, f.n)
    f.close()
    return lz, P, cm, bm, lay, states


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("m,seed", [(1, 1), (5, 2), (40, 3), (300, 4)])
def test_same_results_as_codon_states(prec, m, seed):
    res = synth.residues_dirichlet(m, seed)
    lw = np.random.default_rng(seed).normal(0, 0.5, (m, 6))
    a = _run(res, lw, 0, prec)
    b = _run(res, lw, 1, prec)
    assert b[4] == 1 and a[4] == 0
    tol_z = (1e-6 if prec == 1 else 1e-11) * max(1.0, abs(a[0]))
    assert abs(a[0] - b[0]) <= tol_z
    tol = 1e-5 if prec == 1 else 1e-9
    assert np.abs(a[1] - b[1]).max() <= tol
    assert np.abs(a[2] - b[2]).max() <= tol
    assert np.abs(a[3] - b[3]).max() <= tol
    if m <= 40:
        o = oracle.outside(P0, res, lw, None)
        assert abs(b[0] - o["logZ"]) <= (1e-6 if prec == 1 else 1e-9) * max(1.0, abs(o["logZ"]))
        assert np.abs(b[1] - o["P"]).max() <= (1e-5 if prec == 1 else 2e-7)
        assert np.abs(b[2] - o["codon"]).max() <= 1e-5


def test_state_counts():
    res = [10, 1, 15, 12, 17]  # L, R, S, M, W
    lay, st = _run(res, None, 1, 1)[4:]
    expect = []
    for r in res:
        cods = tm.codon_states(r)
        expect += [len({c[1] for c in cods}), len({(c[1], c[2]) for c in cods}), len({c[3] for c in cods})]
    assert lay == 1 and list(st) == expect
    assert list(st) == [2, 2, 4, 2, 2, 4, 2, 2, 4, 1, 1, 1, 1, 1, 1]
    res = synth.residues_dirichlet(300, 1)
    st = _run(res, None, 1, 1)[5]
    assert 1.5 <= np.mean(st) <= 1.8


def test_tensor_model_same_in_both_layouts():
    cf = _cf()
    V, B, S = synth.tm_params(2, 3, 2)
    model = cf.TensorModel(V, B, S)
    res = synth.residues_dirichlet(20, 5)
    lw = np.random.default_rng(5).normal(0, 0.5, (20, 6))
    out = []
    for layout in (0, 1):
        f = cf.CodonFold(P0)
        cf.cf_set_layout(f.prob, layout)
        f.set_protein(res, lw)
        out.append(f.tm_inside(model, cf.CF_FP64))
        f.close()
    model.close()
    Vn, Bn = tm.normalize(V, B)
    ref = tm.logz(Vn, Bn, S, res, lw)
    assert abs(out[0] - ref) <= 1e-11 * abs(ref) and abs(out[1] - ref) <= 1e-11 * abs(ref)


def test_refusals():
    cf = _cf()
    f = cf.CodonFold(P0)
    cf.cf_set_layout(f.prob, 1)
    with pytest.raises(cf.CFError) as e:
        f.set_protein([1, 2, 3], None, np.zeros((61, 61)))
    assert e.value.status == cf.CF_EINVAL
    f.set_protein([1, 2, 3, 4, 5])
    f.inside(1)
    for call in (lambda: f.sample(4, 1), lambda: f.mfe(), lambda: f.outside(True, True, True),
                 lambda: f.set_weights(None, np.zeros((61, 61)))):
        with pytest.raises(cf.CFError) as e:
            call()
        assert e.value.status == cf.CF_EINVAL
    with pytest.raises(cf.CFError):
        cf.cf_set_layout(f.prob, 2)
    f.close()
