"""CPU oracle for the subsampled-circulant template matcher (see oracle.ftm).

TEST INFRASTRUCTURE. Only the tests, the smoke check of the entry module and
the benchmark's CPU-baseline leg may import this package. The library never
calls it, and it shares no code with the CUDA path.
"""
