"""CPU oracle for the HP-MDR progressive-refactoring hot path.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
CPU-baseline leg of the benchmark.  The product package never imports it.
"""
