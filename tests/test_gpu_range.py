"""Proteins whose composition changes along their length.

The binary32 form keeps one power-of-two exponent per anti-diagonal, and its
far-band tiles rescale by a linear fit of those exponents.  Bands whose
exponents depart too far from the fit are summed term by term: a test hook
forces that path on every band of the 900-nt workload, which must still match
the oracle.  A block of residues that cannot pair (lysines: AAA/AAG) followed
by an ordinary region bends the exponent curve; with a 100-residue block the
strengths of one diagonal's intervals span more than binary32 holds, so the
binary32 form must refuse (CF_ENUMERIC) instead of returning wrong values,
and the binary64 form must match the oracle.
Expected values were written by tests/golden/make_golden.py (oracle only).
"""
from pathlib import Path

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)
GOLD = Path(__file__).resolve().parent / "golden"


def _fold(name):
    import paper_2604_19718_b300 as cf
    res, lw, pb = synth.workload(name)
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    return cf, f


def _golden(name):
    path = GOLD / f"{name}.npz"
    if not path.exists():
        pytest.skip(f"golden {name} not generated")
    return np.load(path)


def test_every_band_summed_term_by_term_matches_oracle():
    """With the tiling bound lowered to zero (test hook), every far band of
    the binary32 inside pass and every outside gather runs term by term with
    exact factors; the 900-nt results must still match the oracle element by
    element."""
    import paper_2604_19718_b300 as cf
    g = _golden("p300_dirichlet")
    res, lw, pb = synth.workload("p300_dirichlet")
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    try:
        cf.cf_debug_set_far_dev_max(0, 0)
        lz = f.inside(cf.CF_FP32_SCALED)
        P, cm, pg = f.outside()
        info = cf.cf_far_band_info(f.prob)
    finally:
        cf.cf_debug_set_far_dev_max(0, cf.FAR_DEV_MAX_DEFAULT)
    f.close()
    nbands = len([d0 for d0 in range(0, 900, 16) if d0 >= 48])
    assert info[1] == nbands and info[3] == 1, info
    assert abs(lz - float(g["logZ"])) <= 1e-6 * abs(float(g["logZ"]))
    assert np.abs(P - g["P"]).max() <= 1e-5
    assert np.abs(cm - g["codon"]).max() <= 1e-5


def test_beyond_binary32_range_is_refused_and_binary64_matches():
    g = _golden("p200_bent")
    cf, f = _fold("p200_bent")
    with pytest.raises(cf.CFError) as e:
        f.inside(cf.CF_FP32_SCALED)
    assert e.value.status == cf.CF_ENUMERIC and "CF_FP64" in str(e.value)
    lz = f.inside(cf.CF_FP64)
    P, cm, pg = f.outside()
    f.close()
    assert abs(lz - float(g["logZ"])) <= 1e-9 * abs(float(g["logZ"]))
    assert np.abs(P - g["P"]).max() <= 2e-7
    assert np.abs(cm - g["codon"]).max() <= 1e-9


def test_ordinary_workloads_stay_tiled():
    """The 300-aa and 1000-aa workloads stay well inside the bound (every far
    band tiled), so their binary32 speed is unaffected by the guard."""
    for name in ("p300_dirichlet", "p1000_weighted"):
        cf, f = _fold(name)
        f.inside(cf.CF_FP32_SCALED)
        f.outside(False, True, False)
        info = cf.cf_far_band_info(f.prob)
        f.close()
        assert info[1] == 0 and info[3] == 0, (name, info)
