"""FP64 CPU oracle for the Para-DPMM split/merge sampler (arXiv 1812.10048).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It
shares no code with the CUDA path (``paper_1812_10048_gb300/csrc``): the two
sides agree only on the written specification of the Philox stream map and
of the algorithm's readings.

Modules
-------
philox    Philox4x32-10 counter-based generator (Salmon et al., SC'11), the
          stream map (tags, counters) and the word -> uniform/Gumbel maps.
dirichlet Log-space Gamma (Marsaglia & Tsang 2000) and Dirichlet draws,
          eq. 28 posteriors of eq. 4 (second line) and eq. 19.
model     Model quantities: the multinomial score of eq. 26, the collapsed
          cluster marginal obtained by integrating eq. 12 against eq. 28, the
          CRP partition probability (eq. 10 read as the standard EPPF) and the
          split / merge Hastings ratios of eq. 7, 14, 16, 23.
sampler   The sampler: eq. 4 blocked sweep with the eq. 8 sub-cluster Gibbs
          step (Section 2.3), and the split / merge moves (Sections 2.3-2.4).
logml     Collapsed log marginal likelihood and its gradient w.r.t. log alpha
          and a gene-wise log beta (derived from eq. 10 and eq. 12).
ari       Adjusted Rand index (Hubert & Arabie 1985), used by Section 3.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against a closed form, a library routine, an
independent algorithm or a statistical law.
"""
