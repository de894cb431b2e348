"""CPU oracle for the GMACO-P route colony -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package. The CUDA library never calls it.
"""
