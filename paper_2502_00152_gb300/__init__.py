"""GB300 (sm_103a) library for deflated HISQ propagator solves.

Method: "Improving HISQ propagator solves using deflation" (LATTICE2024):
even-odd CG on M^dag M with M = D + 2m, thick-restart Lanczos eigenvectors of
the squared massless operator, and deflation with re-deflation (Sections 2, 3).

  paper_2502_00152_gb300.build   -- compiles csrc/*.cu into libhisq.so (nvcc)
  paper_2502_00152_gb300.hisq    -- ctypes binding of include/hisq.h
  paper_2502_00152_gb300.inputs  -- seeded synthetic links and sources

Importing the package loads nothing; the binding loads libhisq.so on first use
and raises if it is missing.
"""
