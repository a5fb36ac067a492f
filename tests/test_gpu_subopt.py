"""Suboptimal configurations (cf_subopt) against brute force: at 2-3 residues
the set of (cost, codon sequence, structure) within the gap equals the
brute-force set over every codon sequence and structure, exactly (integer
costs); at 12-20 residues every returned configuration is valid, its
independently evaluated cost is the reported one and within the gap, none
repeats, the sets grow with the gap, and gap 0 holds the MFE configuration.
tests/bruteforce.py is the independent evaluator."""
import itertools

import numpy as np
import pytest

import bruteforce as bf
import synth

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)


def _fold(res, lw=None, pb=None):
    import paper_2604_19718_b300 as cf
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    return f


def _all_configs(res, lw, pb):
    """(cost, codon ids, partner) of every configuration (brute force)."""
    p = bf.Params(P0)
    opts = [bf.codons_for(r) for r in res]
    out = []
    for combo in itertools.product(*[range(len(o)) for o in opts]):
        cods = [opts[r][combo[r]] for r in range(len(res))]
        cids = [bf.SENSE_ID[c] for c in cods]
        seq = tuple(bf._IDX[b] for c in cods for b in c)
        wc = bf.weight_cost(p, combo, cids, lw, pb)
        for pt in bf.structures(seq):
            e = bf.energy_q(p, seq, pt)
            if e is not None:
                out.append((e + wc, tuple(cids), tuple(int(x) for x in pt)))
    return out


@pytest.mark.parametrize("res,wts,gap", [([3, 17], False, 2.0), ([7, 0, 12], False, 1.5), ([5, 14, 9], True, 2.5),
                                         ([1, 10, 15], True, 0.0)])
def test_equals_bruteforce(res, wts, gap):
    rng = np.random.default_rng(len(res) + int(10 * gap))
    lw = rng.normal(0, 0.5, (len(res), 6)) if wts else None
    pb = rng.normal(0, 0.2, (61, 61)) if wts else None
    allc = _all_configs(res, lw, pb)
    best = min(c[0] for c in allc)
    gq = int(np.floor(gap * 4294967296.0))
    want = sorted(c for c in allc if c[0] <= best + gq)
    f = _fold(res, lw, pb)
    cnt, cost, cod, par = f.subopt(gap, 100000)
    f.close()
    got = sorted((int(cost[i]), tuple(int(x) for x in cod[i]), tuple(int(x) for x in par[i])) for i in range(cnt))
    assert cnt == len(want)
    assert got == want


@pytest.mark.parametrize("m,wts", [(12, False), (20, True)])
def test_valid_unique_and_nested(m, wts):
    res = list(synth.residues_dirichlet(m, m))
    rng = np.random.default_rng(m)
    lw = rng.normal(0, 0.5, (m, 6)) if wts else None
    pb = rng.normal(0, 0.2, (61, 61)) if wts else None
    f = _fold(res, lw, pb)
    q, _, cod0, par0 = f.mfe()
    sets = []
    for gap in (0.0, 0.5, 1.0):
        cnt, cost, cod, par = f.subopt(gap, 20000)
        assert 1 <= cnt <= 20000
        gq = int(np.floor(gap * 4294967296.0))
        keys = set()
        for i in range(cnt):
            assert q <= cost[i] <= q + gq
            assert bf.config_cost(P0, res, cod[i], par[i], lw, pb) == cost[i]
            keys.add((tuple(cod[i]), tuple(par[i])))
        assert len(keys) == cnt  # each configuration once
        sets.append(keys)
    f.close()
    assert (tuple(cod0), tuple(par0)) in sets[0]
    assert sets[0] <= sets[1] <= sets[2]


def test_truncation_and_checks():
    import paper_2604_19718_b300 as cf
    f = _fold([7, 0, 12])
    cnt, cost, cod, par = f.subopt(3.0, 5)
    assert cnt == 6 and len(cost) == 5
    with pytest.raises(cf.CFError) as e:
        f.subopt(-1.0, 5)
    assert e.value.status == cf.CF_EINVAL
    f.close()
