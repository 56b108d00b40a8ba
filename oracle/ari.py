"""Adjusted Rand index (Hubert & Arabie, J. Classification 2, 1985).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 3 of the paper scores clusterings by ARI: the Rand index corrected
for chance, computed from the contingency table n_ij of two labelings with
row sums a_i and column sums b_j:

  ARI = (sum_ij C(n_ij, 2) - E) / (0.5 (sum_i C(a_i, 2) + sum_j C(b_j, 2)) - E),
  E   = sum_i C(a_i, 2) * sum_j C(b_j, 2) / C(n, 2).
"""

import numpy as np


def _pairs(x):
    x = np.asarray(x, dtype=np.float64)
    return (x * (x - 1.0) / 2.0).sum()


def adjusted_rand_index(a, b):
    a = np.unique(np.asarray(a), return_inverse=True)[1]
    b = np.unique(np.asarray(b), return_inverse=True)[1]
    n = a.size
    table = np.zeros((a.max() + 1, b.max() + 1), dtype=np.int64)
    np.add.at(table, (a, b), 1)
    sum_ij = _pairs(table)
    sum_a = _pairs(table.sum(axis=1))
    sum_b = _pairs(table.sum(axis=0))
    expected = sum_a * sum_b / (n * (n - 1) / 2.0)
    denom = 0.5 * (sum_a + sum_b) - expected
    if denom == 0.0:
        return 1.0
    return float((sum_ij - expected) / denom)
