"""Plain FP64 CPU oracle for the batched pair-interaction path.

TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the benchmark's
CPU-baseline leg; never imported by the product package.
"""
