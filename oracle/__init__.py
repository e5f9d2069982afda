"""FP64 CPU oracle of the binary MERA maps (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline and
reference arms of ``bench.py`` may import this package.  It shares no code
with the CUDA library.
"""
