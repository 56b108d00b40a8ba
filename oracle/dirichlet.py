"""Log-space Gamma and Dirichlet draws (oracle side, FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. 4 (second line) and eq. 19 draw each cluster / sub-cluster parameter
vector from its Dirichlet posterior; with the eq. 28 prior and the eq. 26
likelihood that posterior is Dirichlet(lambda + S) where S holds the gene
sums of the cells in the (sub-)cluster.  The first line of eq. 4 draws the
mixing weights from Dirichlet(n_1, ..., n_K, alpha).  A Dirichlet vector is
a normalised vector of independent Gamma variates; with lambda as small as
0.05 the Gamma variates underflow in linear space, so everything is kept in
log space:  log theta_u = log G_u - logsumexp_v log G_v.

Gamma(a) variates follow Marsaglia & Tsang, "A simple method for generating
gamma variables" (ACM TOMS 26(3), 2000): for a >= 1 put d = a - 1/3,
c = 1/sqrt(9d); draw a standard normal z and a uniform u; with v = (1+cz)^3
accept d*v when v > 0 and  log u < z^2/2 + d - d v + d log v.  For a < 1 a
Gamma(a+1) draw G' is boosted:  G = G' * U^(1/a), i.e.
log G = log G' + log(U) / a.

Stream map (see ``oracle/philox.py``): attempt j of element e uses the four
words of Philox counter (e, step, tag<<24|chain, j): words 0 and 1 give the
normal by Box-Muller (z = sqrt(-2 ln u0) cos(2 pi u1)), word 2 the accept
uniform and word 3 the boost uniform of the accepted attempt.  The accept test
is evaluated in the cancellation-free form d*(log1p(e) - e) with e = v - 1.
After MAX_ATTEMPTS rejections (probability below 1e-80) the value log d is
taken.
"""

import numpy as np
from scipy.special import logsumexp

from . import philox

MAX_ATTEMPTS = 64


def log_gamma_draw(shape, seed, chain_id, tag, index, step):
    """log G for G ~ Gamma(shape, 1), one independent draw per element.

    ``shape`` and ``index`` are arrays of equal length; ``index`` is the c0
    word of each element's Philox counters.
    """
    a = np.asarray(shape, dtype=np.float64)
    index = np.asarray(index, dtype=np.int64)
    boost = a < 1.0
    aa = np.where(boost, a + 1.0, a)
    d = aa - 1.0 / 3.0
    c = 1.0 / np.sqrt(9.0 * d)
    out = np.log(d)                       # fallback after MAX_ATTEMPTS
    pending = np.ones(a.shape, dtype=bool)
    for attempt in range(MAX_ATTEMPTS):
        idx = np.nonzero(pending)[0]
        if idx.size == 0:
            break
        w = philox.stream_words(seed, chain_id, tag, index[idx], step, attempt)
        u0 = philox.word_to_uniform(w[:, 0])
        u1 = philox.word_to_uniform(w[:, 1])
        u2 = philox.word_to_uniform(w[:, 2])
        u3 = philox.word_to_uniform(w[:, 3])
        z = np.sqrt(-2.0 * np.log(u0)) * np.cos(2.0 * np.pi * u1)
        y = c[idx] * z
        ok = y > -1.0
        ys = np.where(ok, y, 0.0)
        e = ys * (3.0 + ys * (3.0 + ys))          # v - 1 with v = (1 + y)^3
        accept = ok & (np.log(u2) < 0.5 * z * z + d[idx] * (np.log1p(e) - e))
        logg = np.log(d[idx]) + 3.0 * np.log1p(ys)  # log(d * v)
        logg = np.where(boost[idx], logg + np.log(u3) / np.where(boost[idx], a[idx], 1.0), logg)
        acc = idx[accept]
        out[acc] = logg[accept]
        pending[acc] = False
    return out


def log_dirichlet_draw(conc, seed, chain_id, tag, index0, step):
    """log theta for theta ~ Dirichlet(conc) (1-D ``conc``).

    Element u uses Philox counter word c0 = index0 + u.
    """
    conc = np.asarray(conc, dtype=np.float64)
    logg = log_gamma_draw(conc, seed, chain_id, tag, index0 + np.arange(conc.size), step)
    return logg - logsumexp(logg)
