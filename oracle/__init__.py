"""FP64 CPU oracle for SGD_Tucker (test infrastructure only).

Only the test-suite, the smoke check and the benchmark's CPU-baseline and
reference legs may import this package.  It shares no code with the CUDA path.
"""
