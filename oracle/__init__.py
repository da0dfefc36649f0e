"""FP64 CPU oracle for the total-Lagrangian vectorial LBM (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA library.
"""
