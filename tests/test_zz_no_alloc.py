"""cf_sample_noalloc against cf_sample, through the C ABI.

cf_sample_noalloc is the sampler for callers that cannot allocate device
memory -- code running under a device budget owned by another allocator, or
loops in which cudaMalloc/cudaFree would block or synchronise the device.  Its
scratch is a static device array inside the library.  For the same seed its
samples must equal cf_sample's exactly (integer outputs), on consecutive calls
that reuse the array.  Collected last so that a stopping run has already run
every other test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
P0 = synth.nn_params(0)


@pytest.mark.parametrize("prec", [1, 0])
def test_noalloc_matches_allocating_sampler_on_consecutive_calls(prec):
    import torch

    import paper_2604_19718_b300 as cf
    res, lw, pb = synth.workload("p300_weighted")
    res, lw = res[:80], lw[:80]
    f = cf.CodonFold(P0)
    f.set_protein(res, lw, pb)
    f.inside(prec)
    n, m, N = f.n, f.m, 600  # more samples than the entry point's warps
    for seed in (31, 32):
        ref_c = torch.zeros((N, m), dtype=torch.int32, device="cuda")
        ref_p = torch.zeros((N, n), dtype=torch.int32, device="cuda")
        cf.cf_sample(f.prob, N, seed, ref_c, ref_p)
        out_c = torch.full((N, m), -7, dtype=torch.int32, device="cuda")
        out_p = torch.full((N, n), -7, dtype=torch.int32, device="cuda")
        cf.cf_sample_noalloc(f.prob, N, seed, out_c, out_p)
        torch.cuda.synchronize()
        assert torch.equal(out_c, ref_c)
        assert torch.equal(out_p, ref_p)
    f.close()


def test_noalloc_rejects_host_outputs_and_long_sequences():
    import paper_2604_19718_b300 as cf
    f = cf.CodonFold(P0)
    f.set_protein("MWKLAGHRST" * 3)
    f.inside(1)
    with pytest.raises(cf.CFError) as e:
        cf.cf_sample_noalloc(f.prob, 4, 1, np.zeros((4, f.m), np.int32), np.zeros((4, f.n), np.int32))
    assert e.value.status == cf.CF_EINVAL
    f.set_protein("A" * 1001)  # 3003 nt > CF_NOALLOC_MAX_N
    with pytest.raises(cf.CFError) as e:
        cf.cf_sample_noalloc(f.prob, 4, 1, None, None)
    assert e.value.status == cf.CF_EINVAL and "CF_NOALLOC_MAX_N" in str(e.value)
    f.close()
