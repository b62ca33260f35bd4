"""Plain FP64 CPU oracle for the mirrored-circuit MPO contraction with unswapping.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link or execute
anything here; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA path: the two are independent
implementations of the same method, compared element by element in the parity tests.

Modules:
  mpo         -- the algorithm of the paper (Algorithm 1; Sec. II.B absorption, unswapping,
                 rewiring; Sec. II.C sampling; App. A.1 parallel swap selection; App. A.2
                 non-strict acceptance; App. A.3 adaptive side selection; the Fig. 3
                 telemetry) in plain numpy/scipy FP64, in the paper's order.
  statevector -- brute-force statevector / full-operator simulation used to pin the oracle.

Every function is pinned by tests under ``tests/`` against closed forms, brute force or
invariants (see each function's docstring); functions with no such pin say
"parity unpinned" in their docstring.
"""
