"""The single-codon layout (cf_set_layout(prob, 1), paper Eq. single-tt): the
same protein gives the same log Z, pair probabilities, codon and base
marginals as the codon-state layout and the oracle, in both precisions, with
codon weights; the tensor-based model's log Z is the same in both layouts;
the state counts are the distinct first bases, (first, second) pairs and
third bases, 1.5-1.8 per position; the sampler draws the brute-force
distribution and the oracle's codon marginals in this layout too; the MFE,
its configuration and the suboptimal sets equal those with codon states; the
calls the layout does not serve are refused."""
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


def _layout1_fold(res, lw, prec):
    cf = _cf()
    f = cf.CodonFold(P0)
    cf.cf_set_layout(f.prob, 1)
    f.set_protein(res, lw)
    f.inside(prec)
    return f


@pytest.mark.parametrize("prec", [0, 1])
def test_sampler_exact_distribution(prec):
    """The sampler in the single-codon layout draws (codon sequence,
    structure) with the brute-force probabilities (chi-square, 3 residues
    with codon weights)."""
    import math
    import bruteforce as bf
    res = [1, 15, 10]  # R, S, L: six codons each, the layout's (first, second) pairs differ most
    lw = np.random.default_rng(11).normal(0, 0.5, (3, 6))
    b = bf.summary(P0, res, lw, None)
    probs = {}
    for _, cids, pt, w in b["ensemble"]:
        probs[(cids, pt)] = probs.get((cids, pt), 0.0) + w / b["Z"]
    f = _layout1_fold(res, lw, prec)
    N = 200000
    cod, par = f.sample(N, 17)
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


def test_sampler_marginals_reproducible():
    """30 residues in the single-codon layout: codon frequencies match the
    oracle's marginals within 4.5 sigma, every codon belongs to its residue,
    and the same seed gives the same samples."""
    import math
    res = synth.residues_dirichlet(30, 8)
    lw = np.random.default_rng(8).normal(0, 0.5, (30, 6))
    o = oracle.outside(P0, res, lw, None)
    f = _layout1_fold(res, lw, 1)
    N = 20000
    cod, par = f.sample(N, 5)
    cod2, par2 = f.sample(N, 5)
    f.close()
    assert np.array_equal(cod, cod2) and np.array_equal(par, par2)
    for r in range(len(res)):
        allowed = oracle.codons_of(res[r])
        assert set(np.unique(cod[:, r])) <= set(allowed)
        for s_, cid in enumerate(allowed):
            p = o["codon"][r, s_]
            fr = np.mean(cod[:, r] == cid)
            assert abs(fr - p) <= 4.5 * math.sqrt(p * (1 - p) / N) + 1e-9


@pytest.mark.parametrize("m,seed,gap", [(4, 21, 1.5), (40, 22, 0.3)])
def test_mfe_and_subopt_same_in_both_layouts(m, seed, gap):
    """Integer costs do not depend on which transfer carries a codon's
    weight: the minimum, its configuration and every suboptimal set are the
    same in both layouts."""
    cf = _cf()
    res = synth.residues_dirichlet(m, seed)
    lw = np.random.default_rng(seed).normal(0, 0.5, (m, 6))
    out = {}
    for layout in (0, 1):
        f = cf.CodonFold(P0)
        cf.cf_set_layout(f.prob, layout)
        f.set_protein(res, lw)
        q, kc, cod, par = f.mfe()
        cnt, cost, scod, spar = f.subopt(gap, 5000)
        f.close()
        sub = sorted((int(cost[i]), tuple(int(x) for x in scod[i]), tuple(int(x) for x in spar[i]))
                     for i in range(min(cnt, 5000)))
        out[layout] = (q, tuple(int(x) for x in cod), tuple(int(x) for x in par), cnt, sub)
    assert out[0][0] == out[1][0]
    assert out[0][1:3] == out[1][1:3]
    assert out[0][3] == out[1][3] and out[0][4] == out[1][4]
    assert out[0][3] >= 1


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
    for call in (lambda: f.outside(True, True, True), lambda: f.set_weights(None, np.zeros((61, 61)))):
        with pytest.raises(cf.CFError) as e:
            call()
        assert e.value.status == cf.CF_EINVAL
    with pytest.raises(cf.CFError):
        cf.cf_set_layout(f.prob, 2)
    f.close()
