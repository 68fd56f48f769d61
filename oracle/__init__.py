"""Plain FP64 CPU oracle for the D-VQLS hot path.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import, call, link or run anything in this
package.  It shares no code, header, helper or constant with the CUDA library
in `paper_2604_14435_gb300/`, and it imports nothing from it.

Modules:
  decompose  - FWHT Pauli decomposition, tau pruning, top-L selection and the
               Parseval Frobenius error (Sec. 2.2, Eq. 5, Algorithm 1 Steps 1-2).
  terms      - definition-level states, beta/delta terms, Eq. 1 cost, the
               parameter-shift gradient and the fidelity.
  circuit    - gate-by-gate Hadamard-test circuit simulator on n+1 qubits
               (C, OpenMP over circuits), the primary circuit-level oracle.
  mlp        - FP64 MLP forward/backward for the warm-start gradient checks.
"""
