"""FP64 CPU oracle of the Kino-PAX tree expansion.

TEST INFRASTRUCTURE ONLY.  A plain, slow, double-precision restatement of
the paper's Algorithms 1-4 and Eq. 3-6 that checks the CUDA planner.  Only
the test suite, the package smoke check and the benchmark's CPU-baseline leg
may import it.  It shares no code with the CUDA implementation.
"""
