"""Launch autotuning for a chain or a batch of chains.

The step's kernels take five launch settings (dpmm_set_tuning): statistics
blocks per SM, the dense-tile label kernel's stage count and producer scatter
batch, the parameter-draw blocks per SM and the lanes per cell of the local
Gibbs sub-label kernel (searched only for samplers with local iterations).  None of them changes a result,
so the fastest can be chosen by timing steps of the live sampler itself: its
state is saved before the trials and restored after them (a restored chain
continues bit-identically), and the choice is cached on disk, keyed by the
GPU and the bucketed shape of the workload (genes, clusters, density, cells,
chains), so later samplers of the same shape pay no trials.

Search: coordinate descent from the built-in defaults, one setting at a time
in a fixed order, keeping a candidate only if it is faster by more than the
measurement noise margin.
"""

import json
import math
import os
import time

import numpy as np

CACHE_ENV = "DPMM_TUNING_CACHE"
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1812_10048_gb300",
                             "tuning.json")

# candidate values of each setting, in the order the descent visits them
SEARCH = (
    ("stats_blocks_per_sm", (1, 2, 4, 8)),
    ("tile_stages", (2, 4)),
    ("tile_scatter", (8, 12, 16)),
    ("draw_blocks_per_sm", (1, 2)),
)
# searched only for samplers that run local Gibbs iterations
LOCAL_SEARCH = (("local_stream", (0, 1)), ("local_lanes", (4, 8, 16, 32)))
MARGIN = 0.02          # a candidate must beat the incumbent by 2%


def cache_path(path=None):
    """The cache file: `path`, else $DPMM_TUNING_CACHE, else ~/.cache/..."""
    return path or os.environ.get(CACHE_ENV) or DEFAULT_CACHE


def workload_key(gpu, D, K, density, cells, chains):
    """Bucketed description of a workload: GPU name, D, K rounded up to a
    multiple of 5, density to 0.05, cells to a power of two, chains to a
    power of two."""
    kb = 5 * max(1, math.ceil(max(1, int(K)) / 5))
    db = round(round(float(density) / 0.05) * 0.05, 2)
    nb = 1 << max(0, int(math.ceil(math.log2(max(1, int(cells))))))
    cb = 1 << max(0, int(math.ceil(math.log2(max(1, int(chains))))))
    return f"{gpu}|D={int(D)}|K<={kb}|density~{db:.2f}|cells<={nb}|chains<={cb}"


def load_cache(path=None):
    p = cache_path(path)
    try:
        with open(p) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(key, record, path=None):
    p = cache_path(path)
    os.makedirs(os.path.dirname(p) or ".", exist_ok=True)
    cache = load_cache(p)
    cache[key] = record
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def coordinate_descent(measure, start=None, search=SEARCH, margin=MARGIN):
    """Minimise measure(settings) one setting at a time.

    measure: dict -> seconds per step.  Returns (best settings, best time,
    number of measurements)."""
    best = dict(start or {})
    for name, _ in search:
        best.setdefault(name, 0)
    best_t = measure(dict(best))
    n = 1
    for name, values in search:
        seen = {best[name]}          # the incumbent's value is already measured
        for v in values:
            if v in seen:
                continue
            seen.add(v)
            trial = dict(best)
            trial[name] = v
            t = measure(trial)
            n += 1
            if t < best_t * (1.0 - margin):
                best, best_t = trial, t
    return best, best_t, n


def _chains(sampler):
    """(context, N) of every chain of a Sampler or BatchSampler."""
    if hasattr(sampler, "B"):
        return [(sampler.chain(b), sampler.Ns[b]) for b in range(sampler.B)]
    return [(sampler, sampler.N)]


def _save(sampler):
    saved = []
    for ch, _ in _chains(sampler):
        labels, sub, K, t, m = ch.get_state()
        _, _, sq = ch.stats()
        saved.append((labels, sub, K, t, m, sq))
    return saved


def _restore(sampler, saved):
    for (ch, _), (labels, sub, K, t, m, sq) in zip(_chains(sampler), saved):
        ch.set_state(labels, sub, K, t, m, sq)


def _describe(sampler, indptrs):
    """D, largest K, density, cells and chains of the sampler's workload."""
    chains = _chains(sampler)
    K = max(ch.labels_K() for ch, _ in chains)
    cells = sum(n for _, n in chains)
    nnz = sum(int(ip[-1]) for ip in indptrs)
    density = nnz / max(1, cells * sampler.D)
    return sampler.D, K, density, cells, len(chains)


def gpu_name():
    try:
        import torch
        return torch.cuda.get_device_name().replace("|", "/")
    except Exception:   # the name only labels the cache entry
        return "gpu"


def autotune(sampler, indptrs, *, trial_steps=20, repeats=3, use_cache=True, path=None):
    """Choose and apply the fastest launch settings for `sampler` (a Sampler
    or BatchSampler); `indptrs` are the CSR row pointers of its chain(s)
    (for the density).  Returns a record {"tuning", "ms_per_step",
    "measurements", "source", "key"}; source is "cache" or "measured".  The
    sampler's chain state is unchanged."""
    D, K, density, cells, nch = _describe(sampler, indptrs)
    key = workload_key(gpu_name(), D, K, density, cells, nch)
    if use_cache:
        rec = load_cache(path).get(key)
        if rec is not None:
            _lib_tuning(sampler, rec["tuning"])
            return dict(rec, source="cache", key=key)
    saved = _save(sampler)

    def measure(settings):
        _lib_tuning(sampler, settings)
        times = []
        for _ in range(repeats):
            _restore(sampler, saved)
            sampler.step(2)              # first replay captures the step graph
            sampler.sync()
            t0 = time.perf_counter()
            sampler.step(trial_steps)
            sampler.sync()
            times.append((time.perf_counter() - t0) / trial_steps)
        return float(np.median(times))

    from . import dpmm_get_tuning
    search = SEARCH + (LOCAL_SEARCH if getattr(sampler, "local_iters", 1) > 1 else ())
    best, best_t, n = coordinate_descent(measure, start=dpmm_get_tuning(sampler.ctx),
                                         search=search)
    _restore(sampler, saved)
    _lib_tuning(sampler, best)
    rec = {"tuning": best, "ms_per_step": best_t * 1e3, "measurements": n,
           "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())}
    if use_cache:
        store_cache(key, rec, path)
    return dict(rec, source="measured", key=key)


def _lib_tuning(sampler, settings):
    from . import dpmm_set_tuning
    dpmm_set_tuning(sampler.ctx, **{k: int(v) for k, v in settings.items()})
