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


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Summary of every block the parity tests compared with the oracle (gpu_util.PARITY_LOG):
    per output, the blocks compared and the largest error; and the blocks whose error relative
    to their own norm was above the tolerance but which passed through the absolute lesser /
    greater allowance (energies where those blocks are eta-level differences)."""
    try:
        import gpu_util
    except ImportError:
        return
    log = gpu_util.PARITY_LOG
    if not log:
        return
    tr = terminalreporter
    tr.section("parity summary (CUDA path vs oracle, per block)")
    for tol in sorted({r["tol"] for r in log}):
        tr.write_line(f"tolerance {tol:.0e}:")
        for k in sorted({r["key"] for r in log if r["tol"] == tol}):
            rows = [r for r in log if r["key"] == k and r["tol"] == tol]
            worst = max(r["judged"] for r in rows)
            tr.write_line(f"  {k:8s} blocks {len(rows):6d}  worst judged {worst:.2e}  "
                          f"worst own-norm {max(r['own_rel'] for r in rows):.2e}")
    fl = [r for r in log if r["floor_used"]]
    tr.write_line(f"blocks above the tolerance relative to their own norm, passed by the absolute "
                  f"lesser/greater allowance: {len(fl)} of {len(log)}")
    for r in sorted(fl, key=lambda r: -r["own_rel"])[:10]:
        tr.write_line(f"  {r['test']} {r['key']} energy {r['energy']}: own-norm {r['own_rel']:.2e}, "
                      f"judged {r['judged']:.2e} (tol {r['tol']:.0e})")
