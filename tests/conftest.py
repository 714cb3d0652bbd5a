"""Shared pytest configuration.

Markers: ``gpu`` tests need a CUDA device and the compiled sm_103a library;
everything else runs on the CPU.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def rel_l2(x, ref):
    """sqrt(sum |x - ref|^2 / sum |ref|^2)."""
    import numpy as np
    x = np.asarray(x)
    ref = np.asarray(ref)
    den = np.sum(np.abs(ref) ** 2)
    num = np.sum(np.abs(x - ref) ** 2)
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))
