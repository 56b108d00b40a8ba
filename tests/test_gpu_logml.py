"""Collapsed log marginal likelihood: GPU forward (FP64) / backward (FP32) vs oracle."""

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


def problem(seed=0, N=3000, D=300, K=7):
    from paper_1812_10048_gb300 import synth
    ds = synth.make_dataset(N, D, K, gamma=0.1, lib_mu=np.log(800.0), lib_sigma=0.5, seed=seed)
    rng = np.random.default_rng(seed)
    log_beta = (np.log(0.1) + 0.1 * rng.standard_normal(D)).astype(np.float32)
    return ds, log_beta


def test_forward_and_backward_match_oracle(P):
    import torch
    from oracle.logml import cluster_stats, log_ml, log_ml_grad
    ds, lb = problem()
    K = int(ds.labels.max()) + 2          # one empty cluster index, ignored
    h = P.LogML(ds.indptr, ds.indices, ds.data, ds.N, ds.D, ds.labels, K)
    la = 0.3
    n, S = cluster_stats(ds.indptr, ds.indices, ds.data, ds.N, ds.D, ds.labels, K)
    ref = log_ml(n, S, la, lb.astype(np.float64))
    got = h.forward(la, torch.from_numpy(lb).cuda())
    assert abs(got - ref) <= 1e-10 * abs(ref)
    ga_ref, gb_ref = log_ml_grad(n, S, la, lb.astype(np.float64))
    gb = torch.empty(ds.D, dtype=torch.float32, device="cuda")
    ga = h.backward(la, torch.from_numpy(lb).cuda(), gb)
    torch.cuda.synchronize()
    assert abs(ga - ga_ref) <= 1e-9 * max(1.0, abs(ga_ref))
    np.testing.assert_allclose(gb.cpu().numpy(), gb_ref, rtol=2e-4, atol=1e-3)
    # host pointers work too
    gb_host = np.empty(ds.D, np.float32)
    h.backward(la, lb, gb_host)
    np.testing.assert_allclose(gb_host, gb.cpu().numpy(), rtol=0, atol=0)


def test_autograd_function_matches_finite_differences(P):
    import torch
    ds, lb = problem(seed=1, N=1500, D=120, K=5)
    model = P.LogML(ds.indptr, ds.indices, ds.data, ds.N, ds.D, ds.labels, 5)
    la = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    lbt = torch.from_numpy(lb).cuda().requires_grad_(True)
    out = model(la, lbt)
    out.backward()
    h = 1e-3
    for u in [0, 7, 33, 119]:
        e = np.zeros_like(lb)
        e[u] = h
        fp = model.forward(0.1, torch.from_numpy(lb + e).cuda())
        fm = model.forward(0.1, torch.from_numpy(lb - e).cuda())
        fd = (fp - fm) / (2 * h)
        assert abs(lbt.grad[u].item() - fd) <= 2e-3 * max(1.0, abs(fd))
    # the FP64 forward adds (cluster, gene-block) partials in device order: a
    # step of 1e-6 would sit on its rounding floor (|LML| ~ 1e5, eps ~ 1e-16);
    # 1e-4 keeps the central difference's truncation error below 1e-8
    fa = (model.forward(0.1 + 1e-4, lbt.detach()) - model.forward(0.1 - 1e-4, lbt.detach())) / 2e-4
    assert abs(la.grad.item() - fa) <= 1e-5 * max(1.0, abs(fa))


def test_chain_bound_logml_grad_matches_oracle(P):
    """dpmm_logml_grad on a sampler: the current partition (from the chain's
    statistics) and explicit labels (through the chain's own CSR copy), host
    and device buffers, against the FP64 oracle."""
    import torch
    from oracle.logml import cluster_stats, log_ml, log_ml_grad
    ds, lb = problem(seed=3, N=2500, D=200, K=6)
    s = P.Sampler(ds.indptr, ds.indices, ds.data, ds.N, ds.D, 1.0, 0.5, kmax=32, seed=5)
    s.step(6)
    labels, K = s.labels()
    la = -0.2
    for lab, k, arg in [(labels, K, None), (ds.labels, int(ds.labels.max()) + 1, ds.labels)]:
        n, S = cluster_stats(ds.indptr, ds.indices, ds.data, ds.N, ds.D, lab, k)
        ref = log_ml(n, S, la, lb.astype(np.float64))
        ga_ref, gb_ref = log_ml_grad(n, S, la, lb.astype(np.float64))
        val, ga, gb = P.dpmm_logml_grad(s.ctx, la, lb, labels=arg, K=k)
        assert abs(val - ref) <= 1e-10 * abs(ref)
        assert abs(ga - ga_ref) <= 1e-9 * max(1.0, abs(ga_ref))
        np.testing.assert_allclose(gb, gb_ref, rtol=2e-4, atol=1e-3)
        lbt = torch.from_numpy(lb).cuda()
        argt = None if arg is None else torch.from_numpy(np.ascontiguousarray(arg, np.int32)).cuda()
        val2, ga2, gb2 = P.dpmm_logml_grad(s.ctx, la, lbt, labels=argt, K=k)
        # the FP64 cluster sums are added in device order: equal up to rounding
        assert abs(val2 - val) <= 1e-13 * abs(val)
        assert abs(ga2 - ga) <= 1e-12 * max(1.0, abs(ga))
        np.testing.assert_allclose(gb2, gb, rtol=1e-6, atol=1e-6)
    # the chain itself is untouched
    labels2, K2 = s.labels()
    assert K2 == K and np.array_equal(labels2, labels)
    s.close()


def test_without_counts_only_the_partition_term_remains(P):
    """No cell has a count (T_k = 0, S = 0): the collapsed log ML is the CRP
    partition term K log alpha + lgamma(alpha) - lgamma(alpha + N) + sum_k
    lgamma(n_k) alone, its log-beta gradient vanishes and d/d log alpha =
    K + alpha (psi(alpha) - psi(alpha + N)), in closed form."""
    import torch
    from scipy.special import digamma, gammaln
    N, D, K = 500, 80, 5
    rng = np.random.default_rng(4)
    labels = rng.permutation(np.arange(N) % K).astype(np.int32)
    empty = np.zeros(0, np.int32)
    h = P.LogML(np.zeros(N + 1, np.int32), empty, empty, N, D, labels, K)
    la = 0.4
    a = np.exp(la)
    n = np.bincount(labels, minlength=K)
    ref = K * la + gammaln(a) - gammaln(a + N) + gammaln(n).sum()
    lb = (np.log(0.1) + 0.1 * rng.standard_normal(D)).astype(np.float32)
    got = h.forward(la, torch.from_numpy(lb).cuda())
    assert abs(got - ref) <= 1e-10 * abs(ref)
    gb = torch.empty(D, dtype=torch.float32, device="cuda")
    ga = h.backward(la, torch.from_numpy(lb).cuda(), gb)
    torch.cuda.synchronize()
    ga_ref = K + a * (digamma(a) - digamma(a + N))
    assert abs(ga - ga_ref) <= 1e-9 * max(1.0, abs(ga_ref))
    np.testing.assert_allclose(gb.cpu().numpy(), 0.0, rtol=0, atol=1e-6)
    h.close()
