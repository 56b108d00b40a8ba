"""Seeded synthetic UMI count matrices (cells x genes CSR, int32).

This module only draws inputs; it holds none of the sampler's arithmetic and
is the one piece of code that both the CUDA path's tests and the oracle's
tests use.  It stands in for the 10X datasets of Sections 3-5 (T-cell
subsets, PBMC 68K), which are not available: the data follow the generative
model of Section 2.1 itself -- a mixture of multinomials (eq. 26) whose
gene profiles are Dirichlet draws (eq. 28):

* cluster sizes equal, or proportional to k^(-s) (Zipf s), k = 1..K_true,
  rounded to sum to N (largest remainders);
* profiles theta*_k ~ Dirichlet(gamma * 1_D);
* library sizes l_i = max(1, round(LogNormal(mu, sigma))); optionally a
  fraction of "deep" cells with l_i ~ LogUniform[lo, hi];
* counts x_i ~ Multinomial(l_i, theta*_{c_i}); cells are shuffled.

numpy ``Generator(PCG64(seed))`` drives every draw.
"""

from dataclasses import dataclass

import numpy as np


@dataclass
class Dataset:
    indptr: np.ndarray      # int32 [N+1]
    indices: np.ndarray     # int32 [nnz], sorted within each row
    data: np.ndarray        # int32 [nnz], counts >= 1
    N: int
    D: int
    labels: np.ndarray      # int32 [N], generating cluster of each cell

    @property
    def nnz(self):
        return int(self.indptr[-1])

    @property
    def density(self):
        return self.nnz / float(self.N * self.D) if self.N * self.D else 0.0


def cluster_sizes(N, K, zipf=None):
    w = np.ones(K) if zipf is None else np.arange(1, K + 1, dtype=np.float64) ** (-zipf)
    raw = N * w / w.sum()
    sizes = np.floor(raw).astype(np.int64)
    rem = N - sizes.sum()
    sizes[np.argsort(-(raw - sizes), kind="stable")[:rem]] += 1
    return sizes


def make_dataset(N, D, K_true, *, gamma=0.1, lib_mu=np.log(1500.0), lib_sigma=0.5,
                 zipf=None, deep_frac=0.0, deep_range=(5000.0, 60000.0), seed=1001,
                 chunk=16384, profiles=None):
    """profiles (K_true x D, rows summing to 1) replaces the Dir(gamma) profile draw."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = cluster_sizes(N, K_true, zipf)
    labels = np.repeat(np.arange(K_true), sizes)
    labels = labels[rng.permutation(N)]
    if profiles is None:
        g = rng.gamma(gamma, size=(K_true, D))
        g[g.sum(axis=1) == 0, 0] = 1.0
        profiles = g / g.sum(axis=1, keepdims=True)
    lib = np.maximum(1, np.rint(rng.lognormal(lib_mu, lib_sigma, size=N))).astype(np.int64)
    if deep_frac > 0:
        deep = rng.random(N) < deep_frac
        lo, hi = np.log(deep_range[0]), np.log(deep_range[1])
        lib[deep] = np.rint(np.exp(rng.uniform(lo, hi, size=int(deep.sum())))).astype(np.int64)
    indptr = np.zeros(N + 1, dtype=np.int64)
    idx_parts, val_parts = [], []
    for c0 in range(0, N, chunk):
        c1 = min(N, c0 + chunk)
        dense = np.zeros((c1 - c0, D), dtype=np.int64)
        lab = labels[c0:c1]
        for k in np.unique(lab):
            rows = np.nonzero(lab == k)[0]
            dense[rows] = rng.multinomial(lib[c0 + rows], profiles[k])
        r, c = np.nonzero(dense)
        idx_parts.append(c.astype(np.int32))
        val_parts.append(dense[r, c].astype(np.int32))
        indptr[c0 + 1:c1 + 1] = indptr[c0] + np.cumsum(np.count_nonzero(dense, axis=1))
    indices = np.concatenate(idx_parts) if idx_parts else np.zeros(0, np.int32)
    data = np.concatenate(val_parts) if val_parts else np.zeros(0, np.int32)
    return Dataset(indptr.astype(np.int32), indices, data, int(N), int(D), labels.astype(np.int32))


def _block_counts(args):
    """Counts of one block of cells (a worker of make_dataset_blocks)."""
    seed, b, lab, lib, profiles = args
    rng = np.random.Generator(np.random.PCG64([seed, b + 1]))
    D = profiles.shape[1]
    dense = np.zeros((lab.size, D), dtype=np.int64)
    for k in np.unique(lab):
        rows = np.nonzero(lab == k)[0]
        dense[rows] = rng.multinomial(lib[rows], profiles[k])
    r, c = np.nonzero(dense)
    return (np.count_nonzero(dense, axis=1), c.astype(np.int32), dense[r, c].astype(np.int32))


def _pool(workers):
    import concurrent.futures as cf
    import multiprocessing as mp
    return cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))


def make_dataset_blocks(N, D, K_true, *, gamma=0.1, lib_mu=np.log(1500.0), lib_sigma=0.5,
                        zipf=None, deep_frac=0.0, deep_range=(5000.0, 60000.0), seed=1001,
                        block=65536, workers=None):
    """make_dataset's model for large N: labels, profiles and library sizes from the
    seed's stream, the counts of each block of cells from the stream (seed, block + 1),
    so that blocks can be drawn in parallel (a spawn pool of `workers` processes) and
    the result does not depend on the number of workers."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = cluster_sizes(N, K_true, zipf)
    labels = np.repeat(np.arange(K_true), sizes)
    labels = labels[rng.permutation(N)]
    g = rng.gamma(gamma, size=(K_true, D))
    g[g.sum(axis=1) == 0, 0] = 1.0
    profiles = g / g.sum(axis=1, keepdims=True)
    lib = np.maximum(1, np.rint(rng.lognormal(lib_mu, lib_sigma, size=N))).astype(np.int64)
    if deep_frac > 0:
        deep = rng.random(N) < deep_frac
        lo, hi = np.log(deep_range[0]), np.log(deep_range[1])
        lib[deep] = np.rint(np.exp(rng.uniform(lo, hi, size=int(deep.sum())))).astype(np.int64)
    jobs = [(seed, b, labels[c0:c0 + block], lib[c0:c0 + block], profiles)
            for b, c0 in enumerate(range(0, N, block))]
    if workers is None or workers > 1:
        with _pool(workers) as ex:
            parts = list(ex.map(_block_counts, jobs))
    else:
        parts = [_block_counts(j) for j in jobs]
    indptr = np.zeros(N + 1, dtype=np.int64)
    indptr[1:] = np.cumsum(np.concatenate([p[0] for p in parts]))
    if indptr[-1] >= 2 ** 31:
        raise ValueError("more than 2^31 - 1 non-zeros")
    indices = np.concatenate([p[1] for p in parts])
    data = np.concatenate([p[2] for p in parts])
    return Dataset(indptr.astype(np.int32), indices, data, int(N), int(D), labels.astype(np.int32))


def _one_dataset(kw):
    return make_dataset(**kw)


# Workloads of the sampler, with the shapes of the paper's datasets.
def tiny(seed=1001):
    """2,000 cells x 500 genes, 5 equal clusters, Dir(0.1), LogNormal(log 1500, 0.5)."""
    return make_dataset(2000, 500, 5, gamma=0.1, lib_mu=np.log(1500.0), lib_sigma=0.5, seed=seed)


def pbmc68k(seed=1002):
    """68,000 cells x 1,000 genes (PBMC 68K-sized), 10 Zipf(1.2) clusters, Dir(0.05)."""
    return make_dataset(68000, 1000, 10, gamma=0.05, lib_mu=np.log(1000.0), lib_sigma=0.6,
                        zipf=1.2, seed=seed)


def large(seed=1003, N=1300000, workers=None):
    """1.3M cells x 2,000 genes, 40 Zipf(1.0) clusters, 2% deep cells up to 60,000 UMIs
    (counts drawn block-parallel)."""
    return make_dataset_blocks(N, 2000, 40, gamma=0.05, lib_mu=np.log(1000.0), lib_sigma=0.6,
                               zipf=1.0, deep_frac=0.02, seed=seed, workers=workers)


def batched(B=64, seed=2000, workers=1):
    """B datasets, N_b ~ U[1,000, 50,000], D = 1,000, K_true,b ~ U[3, 20], each from
    make_dataset (seed + b); workers > 1 draws them in a spawn pool."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ns = rng.integers(1000, 50001, size=B)
    Ks = rng.integers(3, 21, size=B)
    kws = [dict(N=int(Ns[b]), D=1000, K_true=int(Ks[b]), gamma=0.1, lib_mu=np.log(1500.0),
                lib_sigma=0.5, seed=seed + b) for b in range(B)]
    if workers is None or workers > 1:
        with _pool(workers) as ex:
            return list(ex.map(_one_dataset, kws))
    return [_one_dataset(kw) for kw in kws]


def similar_types(N, D, K_true, depth, *, sigma=0.05, base_gamma=0.3, seed=1006):
    """Cell types with close expression profiles, for the library-size study: a
    shared base profile ~ Dir(base_gamma) times exp(sigma z_ku) with z standard
    normal per type and gene, renormalised; library sizes LogNormal(log depth,
    0.3).  The profiles do not depend on depth (same seed), so depth alone sets
    how separable the types are."""
    rng = np.random.Generator(np.random.PCG64([seed, 1]))
    base = rng.gamma(base_gamma, size=D)
    base /= base.sum()
    prof = base[None, :] * np.exp(sigma * rng.standard_normal((K_true, D)))
    prof /= prof.sum(axis=1, keepdims=True)
    return make_dataset(N, D, K_true, lib_mu=np.log(depth), lib_sigma=0.3, seed=seed,
                        profiles=prof)


def grad_workload(seed=1005):
    """100,000 cells x 2,000 genes, 25 Zipf(1.0) clusters (labels = generating ones)."""
    return make_dataset(100000, 2000, 25, gamma=0.05, lib_mu=np.log(1000.0), lib_sigma=0.6,
                        zipf=1.0, seed=seed)
