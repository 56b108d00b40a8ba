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


def test_noalloc_matches_the_fp64_oracle(P):
    """Against the oracle's collapsed log ML and analytic gradient (eq. 10 and
    eq. 12 with gene-wise beta), on a non-default stream."""
    import torch
    from oracle.logml import cluster_stats, log_ml, log_ml_grad
    (ds, lb), K, la = problem(23, 2500, 200, 6), 6, 0.2
    n, S = cluster_stats(ds.indptr, ds.indices, ds.data, ds.N, ds.D, ds.labels, K)
    ref = log_ml(n, S, la, lb.astype(np.float64))
    ref_ga, ref_gb = log_ml_grad(n, S, la, lb.astype(np.float64))
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
           for a in (ds.indptr, ds.indices, ds.data, ds.labels)]
    side = torch.cuda.Stream()
    gb = torch.empty(ds.D, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    lml, ga = P.dpmm_logml_grad_noalloc(dev[0], dev[1], dev[2], ds.N, ds.D, dev[3], K, la,
                                        torch.from_numpy(lb).cuda(), gb,
                                        stream=side.cuda_stream)
    assert abs(lml - ref) <= 1e-10 * abs(ref)
    assert abs(ga - ref_ga) <= 1e-9 * max(1.0, abs(ref_ga))
    np.testing.assert_allclose(gb.cpu().numpy(), ref_gb, rtol=2e-4, atol=1e-3)


def test_noalloc_leaves_free_device_memory_unchanged(P):
    """After a first call (which may load the module and its static array),
    further calls change no device memory reservation."""
    import torch
    (ds, lb), K = problem(24, 1200, 100, 3), 3
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
           for a in (ds.indptr, ds.indices, ds.data, ds.labels)]
    lbd = torch.from_numpy(lb).cuda()
    gb = torch.empty(ds.D, dtype=torch.float32, device="cuda")
    P.dpmm_logml_grad_noalloc(dev[0], dev[1], dev[2], ds.N, ds.D, dev[3], K, 0.0, lbd, gb)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        P.dpmm_logml_grad_noalloc(dev[0], dev[1], dev[2], ds.N, ds.D, dev[3], K, 0.0, lbd, gb)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_reports_malformed_inputs(P):
    """Every check precedes the access it guards: a bad label, row, column or
    count is skipped on the device and reported; host memory is refused
    before any launch; a gene total of 2^32 or more is an overflow."""
    import torch
    (ds, lb), K = problem(25, 600, 50, 3), 3
    base = [np.ascontiguousarray(a).copy() for a in (ds.indptr, ds.indices, ds.data, ds.labels)]
    lbd = torch.from_numpy(lb).cuda()
    gb = torch.empty(ds.D, dtype=torch.float32, device="cuda")

    def run(arrs, host_indptr=False):
        dev = [torch.from_numpy(a).cuda() for a in arrs]
        ip = torch.from_numpy(arrs[0]) if host_indptr else dev[0]
        torch.cuda.synchronize()
        return P.dpmm_logml_grad_noalloc(ip, dev[1], dev[2], ds.N, ds.D, dev[3], K, 0.0, lbd, gb)

    run(base)                                        # well formed
    cases = []
    a = [x.copy() for x in base]; a[3][7] = K; cases.append((a, "label outside"))
    a = [x.copy() for x in base]; a[3][9] = -1; cases.append((a, "label outside"))
    a = [x.copy() for x in base]; a[1][11] = ds.D; cases.append((a, "column outside"))
    a = [x.copy() for x in base]; a[2][13] = -4; cases.append((a, "negative count"))
    a = [x.copy() for x in base]
    a[0][5] = a[0][6] + 1; cases.append((a, "malformed indptr"))   # row 5 ends before it starts
    for arrs, msg in cases:
        with pytest.raises(P.DpmmError, match=msg):
            run(arrs)
    with pytest.raises(P.DpmmError, match="device pointers of the current device"):
        run(base, host_indptr=True)
    run(base)                                        # the scratch serves the next call
    # one gene's total over a cluster reaches 2^32: 70,000 cells x 65,535
    n = 70000
    big = [np.arange(n + 1, dtype=np.int32), np.zeros(n, np.int32),
           np.full(n, 65535, np.int32), np.zeros(n, np.int32)]
    dev = [torch.from_numpy(x).cuda() for x in big]
    lb1 = torch.zeros(1, dtype=torch.float32, device="cuda")
    gb1 = torch.empty(1, dtype=torch.float32, device="cuda")
    with pytest.raises(P.DpmmError, match="EOVERFLOW"):
        P.dpmm_logml_grad_noalloc(dev[0], dev[1], dev[2], n, 1, dev[3], 1, 0.0, lb1, gb1)
