"""FP64 CPU oracle (test infrastructure only; never imported by the GPU library).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.
"""
