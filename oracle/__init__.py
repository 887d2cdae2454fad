"""FP64 CPU oracle for the AO/MO vgl path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library; see ``oracle.c`` for what each function computes.
"""
