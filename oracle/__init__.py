"""CPU oracle for the FEF effective-field Fock build (FP64, plain C + NumPy).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import, call or run anything in this package.  It shares no code, header, table or
generator with the CUDA library in ``paper_1708_03377_gb300`` and never imports it.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in ``tests/`` against
closed forms, invariants, brute-force quadrature or library routines (see each test's docstring).
"""
