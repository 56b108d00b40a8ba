"""GB300 Para-DPMM: split/merge sampler for Dirichlet-process mixtures of
multinomials over a cells x genes UMI count matrix (arXiv 1812.10048).

The functions below carry the names of the C ABI in ``include/dpmm.h`` and
only marshal arguments; every step of the sampler runs in libdpmm.so's CUDA
kernels.  ``Sampler`` wraps one context for convenience; ``LogMLFunction``
exposes the collapsed log marginal likelihood to torch.autograd.
"""

import ctypes

import numpy as np

from ._lib import (DpmmError, ENGINE_AUTO, ENGINE_CSR_FP32, ENGINE_TILE_BF16, check, dpmm_opts,
                   dpmm_tuning, lib, ptr)

__all__ = [
    "DpmmError", "Sampler", "LogML", "dpmm_default_opts", "dpmm_init", "dpmm_free", "dpmm_sweep",
    "dpmm_split_merge", "dpmm_step", "dpmm_labels", "dpmm_sync", "dpmm_stream", "dpmm_profile",
    "dpmm_phase_times", "dpmm_plans_applied", "dpmm_debug_engine", "dpmm_set_tuning",
    "dpmm_get_tuning", "TUNING_FIELDS", "dpmm_logml_grad",
    "dpmm_set_hyper",
    "dpmm_eb_step", "empirical_bayes", "dpmm_init_batch",
    "dpmm_chain", "BatchSampler", "dpmm_get_state",
    "dpmm_set_state", "dpmm_get_stats", "dpmm_draw_params", "dpmm_local_gibbs", "dpmm_assign", "dpmm_debug_tile_layout", "dpmm_get_params",
    "dpmm_set_params", "dpmm_debug_scores", "dpmm_debug_tile_scores", "dpmm_debug_moves", "dpmm_logml_create",
    "dpmm_logml_free", "dpmm_logml_forward", "dpmm_logml_backward", "dpmm_logml_grad_noalloc",
    "dpmm_debug_philox",
    "dpmm_debug_curand_philox", "dpmm_debug_tc_gemm", "ENGINE_AUTO", "ENGINE_CSR_FP32", "ENGINE_TILE_BF16",
]


def _i32(a):
    if hasattr(a, "data_ptr"):
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=np.int32)


def dpmm_default_opts(**overrides):
    o = dpmm_opts()
    lib().dpmm_default_opts(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def dpmm_init(indptr, indices, data, N, D, alpha, beta, opts=None, stream=None):
    """Create a chain; arrays may be numpy (host) or torch tensors (host or device)."""
    indptr, indices, data = _i32(indptr), _i32(indices), _i32(data)
    h = ctypes.c_void_p()
    o = opts if opts is not None else dpmm_default_opts()
    check(lib().dpmm_init(ctypes.byref(h), ptr(indptr), ptr(indices), ptr(data), int(N), int(D),
                          float(alpha), float(beta), ctypes.byref(o),
                          ctypes.c_void_p(stream) if stream else None))
    return h


def dpmm_free(ctx):
    lib().dpmm_free(ctx)


def dpmm_init_batch(csrs, Ns, D, alphas, betas, opts=None, stream=None):
    """A batch of chains: csrs = [(indptr, indices, data), ...] (numpy or torch)."""
    B = len(csrs)
    arrs = [tuple(_i32(a) for a in t) for t in csrs]
    P3 = ctypes.c_void_p * B
    ip = P3(*[ptr(a[0]) for a in arrs])
    ix = P3(*[ptr(a[1]) for a in arrs])
    dt = P3(*[ptr(a[2]) for a in arrs])
    n = np.ascontiguousarray(Ns, dtype=np.int64)
    al = np.ascontiguousarray(alphas, dtype=np.float64)
    be = np.ascontiguousarray(betas, dtype=np.float64)
    h = ctypes.c_void_p()
    o = opts if opts is not None else dpmm_default_opts()
    check(lib().dpmm_init_batch(ctypes.byref(h), int(B), ip, ix, dt, ptr(n), int(D), ptr(al),
                                ptr(be), ctypes.byref(o),
                                ctypes.c_void_p(stream) if stream else None))
    return h


def dpmm_chain(ctx, b):
    h = ctypes.c_void_p()
    check(lib().dpmm_chain(ctx, int(b), ctypes.byref(h)))
    return h


def dpmm_sweep(ctx, n_sweeps=1):
    check(lib().dpmm_sweep(ctx, int(n_sweeps)))


def dpmm_split_merge(ctx, mode=0, want_count=True):
    n = ctypes.c_int32(0)
    check(lib().dpmm_split_merge(ctx, int(mode), ctypes.byref(n) if want_count else None))
    return n.value if want_count else None


def dpmm_step(ctx, n_steps=1):
    check(lib().dpmm_step(ctx, int(n_steps)))


def dpmm_labels(ctx, N):
    out = np.empty(int(N), dtype=np.int32)
    K = ctypes.c_int32(0)
    check(lib().dpmm_labels(ctx, ptr(out), ctypes.byref(K)))
    return out, K.value


def dpmm_sync(ctx):
    check(lib().dpmm_sync(ctx))


def dpmm_plans_applied(ctx):
    n = ctypes.c_int64(0)
    check(lib().dpmm_plans_applied(ctx, ctypes.byref(n)))
    return n.value


TUNING_FIELDS = ("stats_blocks_per_sm", "tile_stages", "tile_scatter", "draw_blocks_per_sm",
                 "local_lanes", "local_stream")


def dpmm_set_tuning(ctx, **fields):
    """Launch tuning of a context (see dpmm.h); unnamed fields keep 0 (default)."""
    t = dpmm_tuning()
    for k, v in fields.items():
        if k not in TUNING_FIELDS:
            raise ValueError(f"unknown tuning field {k!r}")
        setattr(t, k, int(v))
    check(lib().dpmm_set_tuning(ctx, ctypes.byref(t)))


def dpmm_get_tuning(ctx):
    """The launch tuning in force, as a dict."""
    t = dpmm_tuning()
    check(lib().dpmm_get_tuning(ctx, ctypes.byref(t)))
    return {k: int(getattr(t, k)) for k in TUNING_FIELDS}


def dpmm_debug_engine(ctx):
    """1 if the chain's latest sweep used the dense-tile engine, else 0."""
    v = ctypes.c_int32(0)
    check(lib().dpmm_debug_engine(ctx, ctypes.byref(v)))
    return int(v.value)


def dpmm_logml_grad(ctx, log_alpha, log_beta, labels=None, K=0, grad=True):
    """Collapsed log marginal likelihood of a sampler's data and its gradient
    w.r.t. (log alpha, log beta): the chain's current partition when labels is
    None, else labels (int32[N], host array or CUDA tensor) in [0, K).
    log_beta: float32[D] host array or CUDA tensor.  Returns
    (logml, d/d log alpha, d/d log beta as float32[D]) or just logml."""
    lb = log_beta if hasattr(log_beta, "data_ptr") else np.ascontiguousarray(log_beta, np.float32)
    lab = None
    if labels is not None:
        lab = labels if hasattr(labels, "data_ptr") else np.ascontiguousarray(labels, np.int32)
    out = ctypes.c_double(0.0)
    ga = ctypes.c_double(0.0)
    D = lb.numel() if hasattr(lb, "numel") else lb.size
    gb = np.zeros(int(D), dtype=np.float32)
    check(lib().dpmm_logml_grad(ctx, ptr(lab) if lab is not None else None, int(K),
                                float(log_alpha), ptr(lb), ctypes.byref(out),
                                ctypes.byref(ga) if grad else None, ptr(gb) if grad else None))
    return (out.value, ga.value, gb) if grad else out.value


def dpmm_set_hyper(ctx, alpha, beta):
    """Replace a chain's alpha and beta between steps (state kept)."""
    check(lib().dpmm_set_hyper(ctx, float(alpha), float(beta)))


def dpmm_eb_step(ctx, eta_alpha, eta_beta, max_step=0.5):
    """One empirical-Bayes step on (log alpha, tied log beta) for the chain's
    current partition; returns (log ML before the step, new alpha, new beta)."""
    lml, a, b = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_double(0.0)
    check(lib().dpmm_eb_step(ctx, float(eta_alpha), float(eta_beta), float(max_step),
                             ctypes.byref(lml), ctypes.byref(a), ctypes.byref(b)))
    return lml.value, a.value, b.value


def empirical_bayes(sampler, rounds, sweeps, eta_alpha, eta_beta, max_step=0.5):
    """Empirical-Bayes loop: `rounds` times, `sweeps` steps of the sampler then
    one dpmm_eb_step.  Returns the trace [(log ML, alpha, beta), ...]."""
    trace = []
    for _ in range(int(rounds)):
        if sweeps:
            sampler.step(int(sweeps))
        trace.append(dpmm_eb_step(sampler.ctx, eta_alpha, eta_beta, max_step))
    return trace


def dpmm_profile(ctx, enable=True):
    check(lib().dpmm_profile(ctx, int(bool(enable))))


def dpmm_phase_times(ctx, n=5):
    out = np.zeros(int(n), dtype=np.float32)
    check(lib().dpmm_phase_times(ctx, ptr(out), int(n)))
    return out


def dpmm_stream(ctx):
    return lib().dpmm_stream(ctx)


def dpmm_get_state(ctx, N):
    labels = np.empty(int(N), dtype=np.int32)
    sub = np.empty(int(N), dtype=np.uint8)
    K, t, m = ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int64(0)
    check(lib().dpmm_get_state(ctx, ptr(labels), ptr(sub), ctypes.byref(K), ctypes.byref(t),
                               ctypes.byref(m)))
    return labels, sub, K.value, t.value, m.value


def dpmm_set_state(ctx, labels, sub, K, t=0, m=0, sumlogq=None):
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    sub = np.ascontiguousarray(sub, dtype=np.uint8)
    sq = None if sumlogq is None else np.ascontiguousarray(sumlogq, dtype=np.float64)
    check(lib().dpmm_set_state(ctx, ptr(labels), ptr(sub), int(K), int(t), int(m), ptr(sq)))


def dpmm_get_stats(ctx, K, D):
    nsub = np.empty((K, 2), dtype=np.uint32)
    Ssub = np.empty((K, 2, D), dtype=np.uint32)
    sumlogq = np.empty(K, dtype=np.float64)
    check(lib().dpmm_get_stats(ctx, ptr(nsub), ptr(Ssub), ptr(sumlogq)))
    return nsub, Ssub, sumlogq


def dpmm_draw_params(ctx):
    check(lib().dpmm_draw_params(ctx))


def dpmm_local_gibbs(ctx, j):
    check(lib().dpmm_local_gibbs(ctx, int(j)))


def dpmm_assign(ctx):
    check(lib().dpmm_assign(ctx))


def dpmm_get_params(ctx, K, D):
    logpi = np.empty(K + 1, dtype=np.float32)
    logtheta = np.empty((3 * K, D), dtype=np.float32)
    check(lib().dpmm_get_params(ctx, ptr(logpi), ptr(logtheta)))
    return logpi, logtheta


def dpmm_set_params(ctx, logpi, logtheta):
    logpi = np.ascontiguousarray(logpi, dtype=np.float32)
    logtheta = np.ascontiguousarray(logtheta, dtype=np.float32)
    check(lib().dpmm_set_params(ctx, ptr(logpi), ptr(logtheta)))


def dpmm_debug_scores(ctx, cells, K):
    cells = np.ascontiguousarray(cells, dtype=np.int32)
    out = np.empty((cells.size, 3 * K), dtype=np.float32)
    check(lib().dpmm_debug_scores(ctx, ptr(cells), int(cells.size), ptr(out)))
    return out


def dpmm_debug_tile_layout(ctx):
    """(T, C, tile_ptr int32[4 T C + 1], tile_ent uint32[n]) of the blocked copy."""
    T, C, n = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int64(0)
    check(lib().dpmm_debug_tile_layout(ctx, ctypes.byref(T), ctypes.byref(C), ctypes.byref(n),
                                       None, None))
    tptr = np.empty(4 * T.value * C.value + 1, dtype=np.int32)
    tent = np.empty(max(1, n.value), dtype=np.uint32)
    check(lib().dpmm_debug_tile_layout(ctx, ctypes.byref(T), ctypes.byref(C), ctypes.byref(n),
                                       ptr(tptr), ptr(tent)))
    return T.value, C.value, tptr, tent[:n.value]


def dpmm_debug_tile_scores(ctx, N, K):
    out = np.empty((int(N), 3 * int(K)), dtype=np.float32)
    check(lib().dpmm_debug_tile_scores(ctx, ptr(out)))
    return out


def dpmm_debug_moves(ctx, kmax):
    chain, n = ctypes.c_int32(0), ctypes.c_int32(0)
    log_h = np.empty(kmax, dtype=np.float64)
    pair_ab = np.empty((kmax, 2), dtype=np.int32)
    check(lib().dpmm_debug_moves(ctx, ctypes.byref(chain), ptr(log_h), ptr(pair_ab),
                                 ctypes.byref(n)))
    return chain.value, log_h[:n.value], pair_ab[:n.value]


def dpmm_logml_create(indptr, indices, data, N, D, labels, K, stream=None):
    indptr, indices, data, labels = _i32(indptr), _i32(indices), _i32(data), _i32(labels)
    h = ctypes.c_void_p()
    check(lib().dpmm_logml_create(ctypes.byref(h), ptr(indptr), ptr(indices), ptr(data), int(N),
                                  int(D), ptr(labels), int(K),
                                  ctypes.c_void_p(stream) if stream else None))
    return h


def dpmm_logml_free(h):
    lib().dpmm_logml_free(h)


def dpmm_logml_forward(h, log_alpha, log_beta):
    out = ctypes.c_double(0.0)
    check(lib().dpmm_logml_forward(h, float(log_alpha), ptr(log_beta), ctypes.byref(out)))
    return out.value


def dpmm_logml_backward(h, log_alpha, log_beta, grad_log_beta):
    ga = ctypes.c_double(0.0)
    check(lib().dpmm_logml_backward(h, float(log_alpha), ptr(log_beta), ctypes.byref(ga),
                                    ptr(grad_log_beta)))
    return ga.value


def dpmm_logml_grad_noalloc(indptr, indices, data, N, D, labels, K, log_alpha, log_beta,
                            grad_log_beta, stream=None):
    """Allocation-free log ML + gradient; CSR and labels must be device tensors.

    Returns (logml, grad_log_alpha) and fills ``grad_log_beta`` (float32[D])."""
    lml, ga = ctypes.c_double(0.0), ctypes.c_double(0.0)
    check(lib().dpmm_logml_grad_noalloc(ptr(indptr), ptr(indices), ptr(data), int(N), int(D),
                                        ptr(labels), int(K), float(log_alpha), ptr(log_beta),
                                        ctypes.byref(lml), ctypes.byref(ga), ptr(grad_log_beta),
                                        ctypes.c_void_p(stream) if stream else None))
    return lml.value, ga.value


def dpmm_debug_philox(ctr, seed):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    check(lib().dpmm_debug_philox(ptr(ctr), int(seed), ptr(out), int(ctr.shape[0])))
    return out


def dpmm_debug_curand_philox(seed, n):
    out = np.empty((int(n), 4), dtype=np.uint32)
    check(lib().dpmm_debug_curand_philox(int(seed), int(n), ptr(out)))
    return out


def dpmm_debug_tc_gemm(A_bf16, B_bf16):
    """C = A B^T on the tensor cores; A uint16[128][Kd], B uint16[N][Kd] (bf16 bits)."""
    A = np.ascontiguousarray(A_bf16, dtype=np.uint16)
    B = np.ascontiguousarray(B_bf16, dtype=np.uint16)
    C = np.empty((128, B.shape[0]), dtype=np.float32)
    check(lib().dpmm_debug_tc_gemm(ptr(A), ptr(B), int(A.shape[1]), int(B.shape[0]), ptr(C)))
    return C


class Sampler:
    """One chain of the sampler on the current CUDA device."""

    def __init__(self, indptr, indices, data, N, D, alpha, beta, *, kmax=256, seed=42,
                 chain_id=0, engine=ENGINE_AUTO, split_q=True, hastings="integrated",
                 open_new_cluster=False, local_iters=1, stream=None):
        self.N, self.D, self.kmax = int(N), int(D), int(kmax)
        self.local_iters = int(local_iters)
        if hastings not in ("integrated", "instantiated"):
            raise ValueError("hastings must be 'integrated' or 'instantiated'")
        opts = dpmm_default_opts(kmax=kmax, seed=seed, chain_id=chain_id, engine=engine,
                                 split_q=int(bool(split_q)),
                                 hastings=int(hastings == "instantiated"),
                                 open_new_cluster=int(bool(open_new_cluster)),
                                 local_iters=int(local_iters))
        self.ctx = dpmm_init(indptr, indices, data, N, D, alpha, beta, opts, stream)

    def close(self):
        if self.ctx is not None:
            dpmm_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1):
        dpmm_sweep(self.ctx, n)

    def split_merge(self, mode=0):
        return dpmm_split_merge(self.ctx, mode)

    def step(self, n=1):
        dpmm_step(self.ctx, n)

    def set_hyper(self, alpha, beta):
        dpmm_set_hyper(self.ctx, alpha, beta)

    def labels(self):
        return dpmm_labels(self.ctx, self.N)

    @property
    def K(self):
        return self.labels_K()

    def labels_K(self):
        K = ctypes.c_int32(0)
        check(lib().dpmm_labels(self.ctx, None, ctypes.byref(K)))
        return K.value

    def get_state(self):
        return dpmm_get_state(self.ctx, self.N)

    def set_state(self, labels, sub, K, t=0, m=0, sumlogq=None):
        dpmm_set_state(self.ctx, labels, sub, K, t, m, sumlogq)

    def stats(self):
        return dpmm_get_stats(self.ctx, self.labels_K(), self.D)

    def sync(self):
        dpmm_sync(self.ctx)

    def plans_applied(self):
        return dpmm_plans_applied(self.ctx)

    @property
    def stream(self):
        return dpmm_stream(self.ctx)


class _ChainView(Sampler):
    """Chain b of a BatchSampler (owned by the batch)."""

    def __init__(self, batch, b, N, D, kmax):
        self.N, self.D, self.kmax = int(N), int(D), int(kmax)
        self.ctx = dpmm_chain(batch.ctx, b)
        self._batch = batch

    def close(self):
        self.ctx = None


class BatchSampler:
    """Independent chains on datasets of uneven size (same D), stepped together:
    one launch per kernel over all chains, one CUDA graph per step."""

    def __init__(self, datasets, D, alpha=1.0, beta=0.5, *, kmax=256, seed=42, chain_id=0,
                 engine=ENGINE_AUTO, split_q=True, hastings="integrated",
                 open_new_cluster=False, local_iters=1, stream=None):
        """datasets: list of (indptr, indices, data, N); alpha / beta scalars or lists."""
        B = len(datasets)
        self.B, self.D, self.kmax = B, int(D), int(kmax)
        self.local_iters = int(local_iters)
        self.Ns = [int(d[3]) for d in datasets]
        al = np.broadcast_to(np.asarray(alpha, dtype=np.float64), (B,))
        be = np.broadcast_to(np.asarray(beta, dtype=np.float64), (B,))
        if hastings not in ("integrated", "instantiated"):
            raise ValueError("hastings must be 'integrated' or 'instantiated'")
        opts = dpmm_default_opts(kmax=kmax, seed=seed, chain_id=chain_id, engine=engine,
                                 split_q=int(bool(split_q)),
                                 hastings=int(hastings == "instantiated"),
                                 open_new_cluster=int(bool(open_new_cluster)),
                                 local_iters=int(local_iters))
        self.ctx = dpmm_init_batch([d[:3] for d in datasets], self.Ns, D, al, be, opts, stream)

    def close(self):
        if self.ctx is not None:
            dpmm_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def chain(self, b):
        return _ChainView(self, b, self.Ns[b], self.D, self.kmax)

    def step(self, n=1):
        dpmm_step(self.ctx, n)

    def sweep(self, n=1):
        dpmm_sweep(self.ctx, n)

    def split_merge(self, mode=0):
        return dpmm_split_merge(self.ctx, mode)

    def sync(self):
        dpmm_sync(self.ctx)

    def plans_applied(self):
        return dpmm_plans_applied(self.ctx)

    @property
    def stream(self):
        return dpmm_stream(self.ctx)


from .autograd import LogML, LogMLFunction  # noqa: E402
