"""FP64 CPU oracle for the PoVar inner solve -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package; the product path never does.
"""
