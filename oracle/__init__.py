"""FP64 CPU oracle for PASD (test infrastructure only).

Nothing on the product path may import this package: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm use it.
"""
