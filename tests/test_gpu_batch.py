"""Batches of small proteins (cf_batch_*): every wavefront kernel covers all
proteins' cells of its diagonal in one launch.  Each protein's results must
equal what a single problem gives for it (same kernels, same inputs: log Z
bit for bit; the binary32 outside's atomic scatters vary below 1e-6) and match
the oracle; lengths from one residue to the batch limit."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)


def _single(res, lw, pb, prec):
    import paper_2604_19718_b300 as cf
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    lz = f.inside(prec)
    P, cm, _ = f.outside(True, True, False)
    f.close()
    return lz, P, cm


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("m,nprot,weights", [(8, 64, False), (8, 37, True), (1, 5, False), (16, 9, True),
                                             (12, 3, False)])
def test_batch_equals_single_problems(prec, m, nprot, weights):
    import paper_2604_19718_b300 as cf
    rng = np.random.default_rng(100 * m + nprot)
    prots = [rng.integers(0, 20, m) for _ in range(nprot)]
    lw = rng.normal(0, 0.5, (nprot, m, 6)) if weights else None
    pb = rng.normal(0, 0.2, (61, 61)) if weights else None
    b = cf.Batch(P0, nprot, m, prec)
    b.set_proteins(prots, lw, pb)
    lz, P, cm = b.run()
    lz2, P2, cm2 = b.run()  # the batch is reusable as it stands
    b.close()
    assert np.array_equal(lz, lz2)
    for k in range(nprot):
        ls, Ps, cms = _single(prots[k], None if lw is None else lw[k], pb, prec)
        assert lz[k] == ls
        assert np.abs(P[k] - Ps).max() <= 1e-6
        assert np.abs(cm[k] - cms).max() <= 1e-6
    for k in range(min(nprot, 4)):  # and against the oracle
        o = oracle.outside(P0, prots[k], None if lw is None else lw[k], pb)
        tol = 1e-6 if prec == 1 else 1e-9
        assert abs(lz[k] - o["logZ"]) <= tol * max(1.0, abs(o["logZ"]))
        assert np.abs(P[k] - o["P"]).max() <= (1e-5 if prec == 1 else 2e-7)
        assert np.abs(cm[k] - o["codon"]).max() <= 1e-5


def test_batch_new_proteins_same_buffers_and_errors():
    """A second set of proteins on the same batch (stale tables cleared),
    and the argument checks."""
    import paper_2604_19718_b300 as cf
    prots = synth.batch_p8(96)
    b = cf.Batch(P0, 48, 8, cf.CF_FP32_SCALED)
    b.set_proteins(prots[:48])
    b.run()
    b.set_proteins(prots[48:])
    lz, P, cm = b.run(pair_prob=False)
    b.close()
    for k in (0, 17, 47):
        ls, _, cms = _single(prots[48 + k], None, None, 1)
        assert lz[k] == ls and np.abs(cm[k] - cms).max() <= 1e-6
    with pytest.raises(cf.CFError) as e:
        cf.Batch(P0, 4, cf_max_m() + 1)
    assert e.value.status == cf.CF_EINVAL
    c = cf.Batch(P0, 2, 3)
    with pytest.raises(cf.CFError) as e:
        c.run()
    assert e.value.status == cf.CF_ESTATE
    with pytest.raises(cf.CFError) as e:
        c.set_proteins(["MWX", "AAA"])
    assert e.value.status == cf.CF_EINVAL
    c.close()


def cf_max_m():
    return 16


def test_batch_input_forms_and_caller_outputs():
    """Residues as letter strings, index lists or one index array give the
    same results; pair probabilities and codon marginals land in the caller's
    arrays (host or device) exactly as in new ones; malformed arrays are
    refused before any launch."""
    import torch

    import paper_2604_19718_b300 as cf
    prots = synth.batch_p8(24)
    idx = np.asarray(prots)
    b = cf.Batch(P0, 24, 8, cf.CF_FP64)
    b.set_proteins([cf.to_letters(p) for p in prots])
    lz, P, cm = b.run()
    b.set_proteins(idx)
    lz2, P2, cm2 = b.run()
    # log Z bit for bit; the outside's binary64 atomic scatters may reorder
    assert np.array_equal(lz, lz2)
    assert np.abs(P - P2).max() <= 1e-12 and np.abs(cm - cm2).max() <= 1e-12
    Ph = np.full_like(P, -1.0)
    cmd = torch.full((24, 8, 6), -1.0, dtype=torch.float64, device="cuda")
    lz3, P3, cm3 = b.run(Ph, cmd)
    assert P3 is Ph and cm3 is cmd
    assert np.array_equal(lz, lz3)
    assert np.abs(P - Ph).max() <= 1e-12 and np.abs(cm - cmd.cpu().numpy()).max() <= 1e-12
    with pytest.raises(ValueError):
        b.run(np.zeros((24, 24, 23), dtype=np.float32))
    with pytest.raises(ValueError):
        b.run(True, np.zeros((24, 8, 6), dtype=np.float32))
    with pytest.raises(ValueError):
        b.set_proteins(np.full((24, 8), 20))
    with pytest.raises(ValueError):
        b.set_proteins(idx[:, :7])
    b.close()
