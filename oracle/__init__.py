"""Plain FP64 CPU oracle of the cell-based FMM gravity solve (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline /
reference legs may import this package.
"""
