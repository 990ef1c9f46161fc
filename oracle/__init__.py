"""Test infrastructure: the FP64 CPU oracle of the OFDM radar receive chain.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg use
this package.  The CUDA library neither imports nor links anything here.
"""
