"""CPU oracle for the BioVSS++ query path: test infrastructure only.

Only the test suite, the smoke check and the benchmark's CPU-baseline leg
may import this package; the product path never does.
"""
