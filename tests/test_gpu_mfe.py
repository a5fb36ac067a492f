"""The GPU minimum free energy (through the C ABI) against the oracle.

Costs are exact integers (2^-32 kcal/mol), so the minimum must equal the
oracle's bit for bit.  Where several configurations attain it, the two
tracebacks may return different ones: the GPU's configuration is checked to
be a valid member of the ensemble whose independently evaluated cost is the
minimum.  The full-size case is compared against the value the oracle wrote
with tests/golden/make_golden.py.
"""
from pathlib import Path

import numpy as np
import pytest

import bruteforce as bf
import oracle
import synth

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)
GOLD = Path(__file__).resolve().parent / "golden"


def _fold():
    import paper_2604_19718_b300 as cf
    return cf.CodonFold(P0)


CASES = {
    "one_residue": ([12], False),
    "two": ([10, 15], False),
    "three": ([0, 1, 2], False),
    "four_weighted": ([5, 7, 2, 14], True),
    "p8_uniform": (list(synth.workload("p8_uniform")[0]), False),
    "p21_weighted": (list(np.random.default_rng(21).integers(0, 20, 21)), True),
    "p47_weighted": (list(np.random.default_rng(47).integers(0, 20, 47)), True),
    "p100": (list(np.random.default_rng(100).integers(0, 20, 100)), False),
}


@pytest.mark.parametrize("name", list(CASES))
def test_mfe_vs_oracle(name):
    res, wts = CASES[name]
    m = len(res)
    rng = np.random.default_rng(m)
    lw = rng.normal(0, 0.5, (m, 6)) if wts else None
    pb = rng.normal(0, 0.2, (61, 61)) if wts else None
    q_o, k_o, _, _ = oracle.mfe(P0, res, lw, pb)
    f = _fold()
    f.set_protein(res, lw, pb)
    q, k, cod, par = f.mfe()
    f.close()
    assert q == q_o
    assert k == k_o
    assert bf.config_cost(P0, res, cod, par, lw, pb) == q


def test_mfe_bruteforce_small():
    res = [3, 17, 8]
    q, _, cod, par = _fold().set_protein(res).mfe()
    assert q == bf.mfe_bruteforce(P0, res)


def test_mfe_full_size_golden_and_weights_update():
    """300 aa / 900 nt with soft weights against the oracle's value; then new
    weights through cf_set_weights (tables kept) against a fresh problem."""
    import paper_2604_19718_b300 as cf
    g = np.load(GOLD / "mfe_p300_weighted.npz")
    res, lw, pb = synth.workload("p300_weighted")
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    q, k, cod, par = f.mfe()
    assert q == int(g["cost"])
    assert bf.config_cost(P0, res, cod, par, lw, pb) == q
    f.set_weights(None, None)
    q0, _, _, _ = f.mfe(traceback=False)
    f.close()
    h = cf.CodonFold(P0)
    h.set_protein(res)
    q1, _, _, _ = h.mfe(traceback=False)
    h.close()
    assert q0 == q1


def test_mfe_bounds_every_sampled_configuration():
    """No configuration drawn by the sampler costs less than the minimum, and
    the minimum is at least the ensemble free energy -kT ln Z."""
    import paper_2604_19718_b300 as cf
    res, lw, pb = synth.workload("p300_weighted")
    res, lw = res[:60], lw[:60]
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    q, k, _, _ = f.mfe(traceback=False)
    lz = f.inside(cf.CF_FP64)
    cod, par = f.sample(64, 9)
    f.close()
    kT = 1.98717e-3 * (P0[180] + 273.15)
    assert -kT * lz <= k + 1e-9
    costs = [bf.config_cost(P0, res, cod[s], par[s], lw, pb) for s in range(64)]
    assert all(c is not None and c >= q for c in costs)


def test_mfe_device_outputs_and_errors():
    import torch

    import paper_2604_19718_b300 as cf
    f = cf.CodonFold(P0)
    with pytest.raises(cf.CFError) as e:
        cf.cf_mfe(f.prob)
    assert e.value.status == cf.CF_ESTATE
    res = CASES["p21_weighted"][0]
    f.set_protein(res)
    q, k, cod, par = f.mfe()
    dc = torch.full((len(res),), -5, dtype=torch.int32, device="cuda")
    dp = torch.full((3 * len(res),), -5, dtype=torch.int32, device="cuda")
    q2, _ = cf.cf_mfe(f.prob, dc, dp)
    torch.cuda.synchronize()
    f.close()
    assert q2 == q
    assert np.array_equal(dc.cpu().numpy(), cod) and np.array_equal(dp.cpu().numpy(), par)
