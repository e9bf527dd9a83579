import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a kernels)")
    config.addinivalue_line("markers", "slow: long CPU-side oracle work")


def rel_fro(x, ref, floor=0.0):
    """Relative Frobenius error ||x - ref||_F / max(||ref||_F, floor)."""
    import numpy as np
    den = max(float(np.linalg.norm(ref)), floor)
    if den == 0.0:
        return float(np.linalg.norm(x))
    return float(np.linalg.norm(x - ref)) / den
