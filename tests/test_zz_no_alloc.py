"""The allocation-free log-ML entry point against the allocating one.

dpmm_logml_grad_noalloc serves callers that cannot allocate device memory
(its scratch is a static device array shared by all calls).  Two calls in a
row, on different problems, must each agree with dpmm_logml_create +
forward + backward within the tolerances of tests/test_gpu_logml.py: the
second call checks that the shared scratch is cleared between calls.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1812_10048_gb300 import build
    build.build()
    import paper_1812_10048_gb300 as P
    return P


def problem(seed, N, D, K):
    from paper_1812_10048_gb300 import synth
    ds = synth.make_dataset(N, D, K, gamma=0.1, lib_mu=np.log(800.0), lib_sigma=0.5, seed=seed)
    rng = np.random.default_rng(seed)
    log_beta = (np.log(0.1) + 0.1 * rng.standard_normal(D)).astype(np.float32)
    return ds, log_beta


def reference(P, ds, K, la, lb):
    import torch
    h = P.LogML(ds.indptr, ds.indices, ds.data, ds.N, ds.D, ds.labels, K)
    lml = h.forward(la, torch.from_numpy(lb).cuda())
    gb = torch.empty(ds.D, dtype=torch.float32, device="cuda")
    ga = h.backward(la, torch.from_numpy(lb).cuda(), gb)
    torch.cuda.synchronize()
    h.close()
    return lml, ga, gb.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_on_two_calls(P):
    import torch
    cases = [(problem(21, 3000, 300, 7), 8, 0.3), (problem(22, 1700, 120, 4), 5, -0.4)]
    for (ds, lb), K, la in cases:
        ref_lml, ref_ga, ref_gb = reference(P, ds, K, la, lb)
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
               for a in (ds.indptr, ds.indices, ds.data, ds.labels)]
        gb = torch.full((ds.D,), float("nan"), dtype=torch.float32, device="cuda")
        lml, ga = P.dpmm_logml_grad_noalloc(dev[0], dev[1], dev[2], ds.N, ds.D, dev[3], K, la,
                                            torch.from_numpy(lb).cuda(), gb)
        assert abs(lml - ref_lml) <= 1e-10 * abs(ref_lml)
        assert abs(ga - ref_ga) <= 1e-9 * max(1.0, abs(ref_ga))
        np.testing.assert_allclose(gb.cpu().numpy(), ref_gb, rtol=2e-4, atol=1e-3)


def test_noalloc_rejects_sizes_beyond_its_static_scratch(P):
    import torch
    z = torch.zeros(8, dtype=torch.int32, device="cuda")
    lb = torch.zeros(2048, dtype=torch.float32, device="cuda")
    gb = torch.zeros(2048, dtype=torch.float32, device="cuda")
    with pytest.raises(P.DpmmError, match="K \\* D <= 1048576"):
        P.dpmm_logml_grad_noalloc(z, z, z, 2, 2048, z, 1024, 0.0, lb, gb)
