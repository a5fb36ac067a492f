"""Failure paths of the C ABI, driven without faulting the GPU.

A bounded device wait is made to give up at once (a test hook lowers its
poll limit to zero: every kernel that waits for staged inputs records the
timeout, still waits for its own copies and returns), and a device
allocation is made to fail on the host (a test hook in the library's
allocator).  Each call must report its status, and the same problem must then
give correct results once the hook is off.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)


def _cf():
    import paper_2604_19718_b300 as cf
    return cf


def _case(m=40):
    res, lw, pb = synth.workload("p300_weighted")
    return res[:m], lw[:m], pb


@pytest.mark.parametrize("prec", [1, 0])
def test_wait_timeout_then_reuse(prec):
    cf = _cf()
    res, lw, pb = _case()
    o = oracle.outside(P0, res, lw, pb)
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    try:
        cf.cf_debug_set_wait_polls(0, 0)
        with pytest.raises(cf.CFError) as e:
            f.inside(prec)
        assert e.value.status == cf.CF_ETIMEOUT
        with pytest.raises(cf.CFError) as e:  # no inside result survives the failure
            f.outside()
        assert e.value.status == cf.CF_ESTATE
        cf.cf_debug_set_wait_polls(0, cf.WAIT_POLLS_DEFAULT)
        lz = f.inside(prec)
        cf.cf_debug_set_wait_polls(0, 0)
        with pytest.raises(cf.CFError) as e:
            f.outside()
        assert e.value.status == cf.CF_ETIMEOUT
    finally:
        cf.cf_debug_set_wait_polls(0, cf.WAIT_POLLS_DEFAULT)
    P, cm, pg = f.outside()
    f.close()
    tol = 1e-6 if prec == 1 else 1e-9
    assert abs(lz - o["logZ"]) <= tol * max(1.0, abs(o["logZ"]))
    assert np.abs(P - o["P"]).max() <= 1e-5
    assert np.abs(cm - o["codon"]).max() <= 1e-5


def test_tm_wait_timeout_then_reuse():
    """The tensor-model cell kernel's bounded waits for its staged blocks."""
    from oracle import tensor_model as tm
    cf = _cf()
    V, B, S = synth.tm_params(1, 3, 2)
    res = [4, 12, 0, 17, 9, 2]
    model = cf.TensorModel(V, B, S)
    f = cf.CodonFold(P0)
    f.set_protein(res)
    try:
        cf.cf_debug_set_wait_polls(0, 0)
        for prec in (cf.CF_FP32_SCALED, cf.CF_FP64):
            with pytest.raises(cf.CFError) as e:
                f.tm_inside(model, prec)
            assert e.value.status == cf.CF_ETIMEOUT
    finally:
        cf.cf_debug_set_wait_polls(0, cf.WAIT_POLLS_DEFAULT)
    Vn, Bn = tm.normalize(V, B)
    ref = tm.logz(Vn, Bn, S, res)
    assert abs(f.tm_inside(model, cf.CF_FP64) - ref) <= 1e-11 * abs(ref)
    f.close()
    model.close()


def test_tm_wait_timeout_in_clusters_then_reuse():
    """The same at 150 nt, where the longest lengths split each cell over
    clusters of 2, 4 and 8 CTAs: every CTA of a cluster leaves through both
    cluster barriers, and the problem then gives its earlier log Z exactly."""
    cf = _cf()
    V, B, S = synth.tm_params(2, 4, 2)
    res = synth.residues_dirichlet(50, 6)
    model = cf.TensorModel(V, B, S)
    f = cf.CodonFold(P0)
    f.set_protein(res)
    ref = {prec: f.tm_inside(model, prec) for prec in (cf.CF_FP32_SCALED, cf.CF_FP64)}
    try:
        cf.cf_debug_set_wait_polls(0, 0)
        for prec in (cf.CF_FP32_SCALED, cf.CF_FP64):
            with pytest.raises(cf.CFError) as e:
                f.tm_inside(model, prec)
            assert e.value.status == cf.CF_ETIMEOUT
    finally:
        cf.cf_debug_set_wait_polls(0, cf.WAIT_POLLS_DEFAULT)
    for prec in (cf.CF_FP32_SCALED, cf.CF_FP64):
        assert f.tm_inside(model, prec) == ref[prec]
    f.close()
    model.close()


def test_forced_allocation_failures_leave_problem_usable():
    cf = _cf()
    res, lw, pb = _case()
    o = oracle.outside(P0, res, lw, pb)
    f = cf.CodonFold(P0)
    try:
        # cf_set_protein: the first device allocation fails
        cf.cf_debug_fail_alloc(0)
        with pytest.raises(cf.CFError) as e:
            f.set_protein(res, lw, pb)
        assert e.value.status == cf.CF_ENOMEM
        with pytest.raises(cf.CFError) as e:  # no protein is left behind
            f.inside(1)
        assert e.value.status == cf.CF_ESTATE
        cf.cf_debug_fail_alloc(-1)
        f.set_protein(res, lw, pb)
        # cf_inside: an allocation in the middle of the tables fails
        cf.cf_debug_fail_alloc(5)
        with pytest.raises(cf.CFError) as e:
            f.inside(1)
        assert e.value.status == cf.CF_ENOMEM
        cf.cf_debug_fail_alloc(-1)
        lz = f.inside(1)
        # cf_outside: the adjoint tables do not fit; the precision's tables go
        cf.cf_debug_fail_alloc(3)
        with pytest.raises(cf.CFError) as e:
            f.outside()
        assert e.value.status == cf.CF_ENOMEM
        with pytest.raises(cf.CFError) as e:
            f.outside()
        assert e.value.status == cf.CF_ESTATE
        cf.cf_debug_fail_alloc(-1)
        lz2 = f.inside(1)
        P, cm, pg = f.outside()
        # the sampler's scratch
        cf.cf_debug_fail_alloc(0)
        with pytest.raises(cf.CFError) as e:
            f.sample(16, 3)
        assert e.value.status == cf.CF_ENOMEM
        cf.cf_debug_fail_alloc(-1)
        cod, par = f.sample(16, 3)
    finally:
        cf.cf_debug_fail_alloc(-1)
    f.close()
    assert lz == lz2
    assert abs(lz - o["logZ"]) <= 1e-6 * max(1.0, abs(o["logZ"]))
    assert np.abs(P - o["P"]).max() <= 1e-5 and np.abs(cm - o["codon"]).max() <= 1e-5
    assert (cod >= 0).all() and cod.shape == (16, len(res))


def test_pinned_host_outputs_rejected_by_noalloc_sampler():
    """Pinned host memory is host memory: the no-allocation sampler, which
    writes its outputs in place, rejects it before any launch."""
    import torch
    cf = _cf()
    f = cf.CodonFold(P0)
    f.set_protein("MWKLAGHRST" * 3)
    f.inside(1)
    c = torch.zeros((4, f.m), dtype=torch.int32).pin_memory()
    q = torch.zeros((4, f.n), dtype=torch.int32).pin_memory()
    with pytest.raises(cf.CFError) as e:
        cf.cf_sample_noalloc(f.prob, 4, 1, c, q)
    assert e.value.status == cf.CF_EINVAL
    f.close()
