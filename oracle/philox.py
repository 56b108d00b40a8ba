"""Philox4x32-10 and the sampler's random-stream map (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): a 4-word
counter and a 2-word key pass through 10 rounds; each round multiplies
counter words 0 and 2 by fixed odd constants, takes the high and low halves
of the 64-bit products and mixes them with words 1 and 3 and the key; the key
is advanced by two Weyl constants between rounds.

Every random quantity of the sampler is one Philox call on a counter built
from the stream map below, so the oracle and the CUDA path draw identical
words without sharing code.  Counter layout::

    (c0, c1, c2, c3) = (index, step, (tag << 24) | chain_id, j)

with key = (seed & 0xffffffff, seed >> 32).  Tags:

    TAG_LABEL      0  eq. 4 label Gumbels: c0 = cell i, c1 = sweep t,
                      c3 = k // 4, word k % 4 for cluster k
    TAG_SUBLABEL   1  eq. 8 sub-label Gumbels: c0 = i, c1 = t, c3 = 0,
                      words 0, 1 for r = 0, 1
    TAG_THETA      2  eq. 4 / eq. 19 Gamma draws: c0 = row * D + u,
                      c1 = t, c3 = attempt
    TAG_PI         3  eq. 4 mixing-weight Gamma draws: c0 = k, c1 = t,
                      c3 = attempt
    TAG_MOVE       4  split/merge chain coin (c0 = 0) and split accept
                      (c0 = k + 1): c1 = call m, c3 = 0, word 0
    TAG_PAIR       5  merge pairing keys: c0 = k, c1 = m, c3 = 0, word 0
    TAG_MERGE      6  merge accept: c0 = lower cluster index, c1 = m, word 0
    TAG_SUBINIT    7  random sub-label (re)initialisation, word 0:
                      c3 = 0 at init (c1 = 0), 1 for the empty-sub-cluster
                      reset of sweep t (c1 = t), 2 after a split in call m
                      (c1 = m)

Local Gibbs iterations j = 1, 2, .. after sweep t (Section 2.3; more than one
only when asked for) use their own tags, c1 = t:

    16 + 2 (j - 1)  eq. 19 sub-cluster Gamma draws: c0 = row * D + u with
                    row = 3k + 1 + r, c3 = attempt
    17 + 2 (j - 1)  eq. 8 sub-label Gumbels: c0 = i, c3 = 0, words 0, 1

A 32-bit word w maps to the uniform ``((w >> 9) + 0.5) * 2**-23``, which lies
in (0, 1) and is exactly representable in both FP32 and FP64, so both sides
see the same uniform.
"""

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
ROUNDS = 10

TAG_LABEL = 0
TAG_SUBLABEL = 1
TAG_THETA = 2
TAG_PI = 3
TAG_MOVE = 4
TAG_PAIR = 5
TAG_MERGE = 6
TAG_SUBINIT = 7

LOCAL_TAG0 = 16
LOCAL_MAX_ITERS = 16


def tag_local_theta(j):
    """Tag of the sub-cluster Gamma draws of local Gibbs iteration j >= 1."""
    return LOCAL_TAG0 + 2 * (j - 1)


def tag_local_sub(j):
    """Tag of the sub-label Gumbels of local Gibbs iteration j >= 1."""
    return LOCAL_TAG0 + 2 * (j - 1) + 1


SUBINIT_INIT = 0
SUBINIT_RESET = 1
SUBINIT_SPLIT = 2


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four output words of Philox4x32-10 (broadcast over arrays)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint32) for v in np.broadcast_arrays(
        np.asarray(c0, dtype=np.uint64) & 0xFFFFFFFF, np.asarray(c1, dtype=np.uint64) & 0xFFFFFFFF,
        np.asarray(c2, dtype=np.uint64) & 0xFFFFFFFF, np.asarray(c3, dtype=np.uint64) & 0xFFFFFFFF))
    k0 = np.uint32(int(k0) & 0xFFFFFFFF)
    k1 = np.uint32(int(k1) & 0xFFFFFFFF)
    with np.errstate(over="ignore"):
        for r in range(ROUNDS):
            if r > 0:
                k0 = np.uint32((int(k0) + int(W0)) & 0xFFFFFFFF)
                k1 = np.uint32((int(k1) + int(W1)) & 0xFFFFFFFF)
            p0 = M0 * c0.astype(np.uint64)
            p1 = M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & np.uint64(0xFFFFFFFF)).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & np.uint64(0xFFFFFFFF)).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack([c0, c1, c2, c3], axis=-1)


def stream_words(seed, chain_id, tag, index, step, j):
    """Philox words for the stream map: counter (index, step, tag<<24|chain, j)."""
    seed = int(seed)
    c2 = ((int(tag) & 0xFF) << 24) | (int(chain_id) & 0xFFFFFF)
    return philox4x32_10(index, step, c2, j, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def word_to_uniform(w):
    """u = ((w >> 9) + 0.5) * 2**-23, in (0, 1), exact in FP32 and FP64."""
    w = np.asarray(w, dtype=np.uint32)
    return ((w >> np.uint32(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def uniform_to_gumbel(u):
    """Standard Gumbel variate -log(-log u)."""
    return -np.log(-np.log(u))
