"""Plain FP64 CPU oracle of the auxiliary Kalman sampler.

TEST INFRASTRUCTURE, not part of the library. Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it. It shares no code with the CUDA path:
it takes its inputs (model, data, seeds) as arguments and implements its
own Philox generator.

Modules:
  philox  Philox4x32-10 + Box-Muller streams (Salmon et al. 2011).
  kalman  Kalman filter and RTS sampler algorithms (Appendix A.1), parallel-filter
          elements and operator (Appendix A.2.1), (G, U) backward scan
          (Eqs. (A.14)-(A.15), Proposition A.1), Hillis-Steele scan (Appendix A.2.1).
  mcmc    one auxiliary Kalman MH step (Alg. 2, first-order, Gaussian
          dynamics) with the direct-formula acceptance ratio.
  dense   brute-force stacked-path Gaussian (Eq. (2.2)) for tiny T·d.
  bridging  divide-and-conquer (bridging) pathwise sampler (Section 2.4.2,
          Appendix A.2.3).
  sqrt_filter  square-root form of the parallel filter (the fix Section 4.1
          names for its single-precision divergence).
"""
