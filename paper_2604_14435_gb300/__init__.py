"""GB300-native D-VQLS hot path: FWHT Pauli decomposition with tau pruning and
the batched Hadamard-test term evaluation (cost and parameter-shift gradient),
as hand-written sm_103a CUDA behind a C-ABI (include/dvqls.h).

`dvqls` is the thin ctypes binding of that library; `workloads` builds the
seeded synthetic inputs.  Importing the package loads nothing; the CUDA
library is opened on first use and its absence is an error.
"""
__all__ = ["dvqls", "workloads"]
