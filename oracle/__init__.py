"""FP64 CPU oracle of the deflated HISQ propagator solve -- test infrastructure.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg use
this package; the CUDA library never imports it.  See oracle.py.
"""
