"""GB300-native (sm_103a) split-step Fourier / Crank-Nicolson z-step library.

The compute path is the CUDA shared library built from ``csrc/`` and called
through its C-ABI (``include/fcn.h``) by the thin ctypes binding in
``paper_1507_05988_gb300.fcn``.  Importing this package does not load the
library; ``paper_1507_05988_gb300.fcn`` does, and fails loudly if it is
missing.
"""

__all__ = ["fcn", "workloads"]
