"""FP64 CPU oracle for the extrapolated GBS macro-step (Ellison & Fornberg,
"A parallel-in-time approach for wave-type PDEs", arXiv 1907.11771).

This package is TEST INFRASTRUCTURE.  It is a plain, slow, deliberately
unoptimised restatement of what the paper defines, written so that a reader
can check it against the paper by eye:

* ``weights``  -- exact rational extrapolation weights (Sec. 3.2 eq. "vander",
  Sec. 3.7 eqs. "order_constraints"/"cdep_computation"), the stability
  polynomial R(xi) = sum_k c_k P_k(xi) (Appendix A, Appendix B) and the
  imaginary stability boundary ISB by exact root isolation (Sec. 2.2).
* ``mol``      -- the method-of-lines right-hand sides: periodic centred
  finite differences of order 4 and 6, the 1D wave system and 2D/3D
  acoustics, and their transposes (needed by the adjoint).
* ``gbs``      -- one GBS sequence (Sec. 2.1 eq. "GBS": Forward Euler start,
  N leap-frog steps, averaging), the extrapolated macro-step
  sum_k c_k y*_k (Sec. 2.1, Sec. 3.2), the discrete adjoint of that
  macro-step and the receiver misfit.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code, constants or tables with it.
"""
