"""The autograd wrapper on the GPU: gradients of log Z through cf_inside /
cf_outside against the oracle's marginals and against central finite
differences (h = 1e-4, FP64) of the GPU's own log Z; weight updates through
cf_set_weights; the weight ascent on the 300-aa soft-weighted protein."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)
TOL = {0: 1e-9, 1: 1e-5}  # marginals, FP64 / FP32 scaled


def _fold(res, lw=None, pb=None):
    import paper_2604_19718_b300 as cf
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    return f


@pytest.mark.parametrize("prec", [0, 1])
def test_autograd_equals_oracle_marginals(prec):
    from paper_2604_19718_b300 import adjoint
    res, lw, pb = synth.workload("p300_weighted")
    res, lw = res[:40], lw[:40]
    f = _fold(res)
    lw_t = torch.tensor(lw, device="cuda", requires_grad=True)
    pb_t = torch.tensor(pb, device="cuda", requires_grad=True)
    z = adjoint.LogZ.apply(lw_t, pb_t, f, prec)
    z.backward()
    o = oracle.outside(P0, res, lw, pb)
    assert abs(float(z.detach()) - o["logZ"]) <= 1e-6 * max(1.0, abs(o["logZ"]))
    assert np.abs(lw_t.grad.cpu().numpy() - o["codon"]).max() < TOL[prec]
    assert np.abs(pb_t.grad.cpu().numpy() - o["pair_grad"]).max() < TOL[prec] * 10
    f.close()


def test_set_weights_equals_fresh_protein():
    """Updating weights in place gives the same log Z and marginals as a
    problem built from scratch with those weights."""
    res, lw, pb = synth.workload("p300_weighted")
    res, lw = res[:60], lw[:60]
    a = _fold(res)
    a.inside(1)
    a.set_weights(lw, pb)
    za = a.inside(1)
    _, ca, ga = a.outside(False)
    b = _fold(res, lw, pb)
    zb = b.inside(1)
    _, cb, gb = b.outside(False)
    # the inside pass has no atomics (bitwise equal); the FP32 outside adds with
    # atomics in varying order, far below its 1e-5 tolerance against the oracle
    assert za == zb and np.abs(ca - cb).max() < 1e-7 and np.abs(ga - gb).max() < 1e-7
    import paper_2604_19718_b300 as cf
    a.set_weights(lw * 0, None)
    with pytest.raises(cf.CFError) as e:
        a.outside()  # weights changed: the inside pass is stale
    assert e.value.status == cf.CF_ESTATE
    bad = lw.copy()
    bad[3, 0] = np.nan
    with pytest.raises(cf.CFError) as e:
        a.set_weights(bad, None)
    assert e.value.status == cf.CF_EINVAL
    a.close()
    b.close()


def test_central_differences_full_size():
    """300-aa protein, all weights on: sampled coordinates of the gradient
    against (logZ(w + h e) - logZ(w - h e)) / 2h in FP64 on the GPU."""
    from paper_2604_19718_b300 import adjoint
    res, lw, pb = synth.workload("p300_weighted")
    f = _fold(res, lw, pb)
    lw_t = torch.tensor(lw, device="cuda", requires_grad=True)
    pb_t = torch.tensor(pb, device="cuda", requires_grad=True)
    adjoint.LogZ.apply(lw_t, pb_t, f, 0).backward()
    g_lw, g_pb = lw_t.grad.cpu().numpy(), pb_t.grad.cpu().numpy()
    mask = adjoint.slot_mask(synth.to_string(res))
    rng = np.random.default_rng(5)
    h = 1e-4

    def logz(lw_, pb_):
        f.set_weights(lw_, pb_)
        return f.inside(0)
    valid = np.argwhere(mask)
    for r, s in valid[rng.choice(len(valid), 5, replace=False)]:
        e = np.zeros_like(lw)
        e[r, s] = h
        fd = (logz(lw + e, pb) - logz(lw - e, pb)) / (2 * h)
        assert abs(fd - g_lw[r, s]) < 1e-6, (r, s, fd, g_lw[r, s])
    used = np.argwhere(g_pb > 0.05)
    for c1, c2 in used[rng.choice(len(used), 4, replace=False)]:
        e = np.zeros_like(pb)
        e[c1, c2] = h
        fd = (logz(lw, pb + e) - logz(lw, pb - e)) / (2 * h)
        assert abs(fd - g_pb[c1, c2]) < 1e-6, (c1, c2, fd, g_pb[c1, c2])
    f.close()


def test_ascent_trajectory_equals_oracle():
    """Three ascent steps on a 30-aa prefix: the GPU (FP64) and the oracle
    produce the same weights."""
    from paper_2604_19718_b300 import adjoint
    res, _, pb = synth.workload("p300_weighted")
    res = res[:30]
    aa = synth.to_string(res)
    fstar = adjoint.frequency_targets(aa, synth.ascent_targets(300)[:30])
    f = _fold(res)
    lw_gpu, hist = adjoint.weight_ascent(f, aa, fstar, steps=3, pb=pb, precision=0, device="cuda")
    lw = np.zeros((30, 6))
    for _ in range(3):
        p = oracle.outside(P0, res, lw, pb)["codon"]
        lw = lw + np.where(adjoint.slot_mask(aa), fstar - p, 0.0)
    assert np.abs(lw_gpu.cpu().numpy() - lw).max() < 1e-9
    f.close()


def test_weight_ascent_config3():
    """50 steps at 300 aa in FP32: the objective rises and the largest
    frequency gap shrinks."""
    from paper_2604_19718_b300 import adjoint
    res, lw0, pb = synth.workload("p300_weighted")
    aa = synth.to_string(res)
    fstar = adjoint.frequency_targets(aa, synth.ascent_targets(300))
    f = _fold(res)
    _, hist = adjoint.weight_ascent(f, aa, fstar, steps=50, lw0=lw0, pb=pb, device="cuda")
    obj = [h["objective"] for h in hist]
    gaps = [h["max_gap"] for h in hist]
    assert all(b >= a - 1e-3 for a, b in zip(obj, obj[1:]))
    assert gaps[-1] < 0.1 * gaps[0]
    f.close()
