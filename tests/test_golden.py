"""Stored expected values (tests/golden/, written by tests/golden/make_golden.py from the oracle
only): the oracle must keep reproducing them (CPU), and the CUDA path must match them block by
block (GPU) without running the oracle, under the stored per-energy floors at the FP64
tolerance."""
import json
import os

import numpy as np
import pytest

import oracle
from gpu_util import TOL_FP64, block_errors

HERE = os.path.dirname(os.path.abspath(__file__))
KEYS = ("R_diag", "R_upper", "R_lower", "L_diag", "L_upper", "G_diag", "G_upper")


def load():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(HERE, "golden", "random_3x4.json")) as f:
        d = json.load(f)
    blocks = {k: np.array(v)[..., 0] + 1j * np.array(v)[..., 1] for k, v in d["blocks"].items()}
    return mod.system(), d, blocks


def test_golden_oracle_reproduces_stored_values():
    s, d, blocks = load()
    assert np.array_equal(s.energies, np.array(d["energies"]))
    for e in range(len(s.energies)):
        ref = oracle.solve_g(s, e, surface="eig")
        for k in KEYS:
            errs = block_errors(ref[k], blocks[k][e], abs_floor=d["lesser_abs_floor"][e] if k[0] in "LG" else 0.0)
            assert errs.max() <= 1e-12, (k, e, errs.max())


def test_golden_fixture_invariants():
    """The stored blocks themselves satisfy what the definitions fix: lesser/greater diagonal
    blocks anti-Hermitian (Sec. 5.2 symmetrisation), -i G^< and i G^> positive semidefinite,
    spectral function i (G^R - G^A) positive semidefinite on the diagonal."""
    _, _, blocks = load()
    for e in range(blocks["R_diag"].shape[0]):
        for i in range(blocks["R_diag"].shape[1]):
            L, G, R = blocks["L_diag"][e, i], blocks["G_diag"][e, i], blocks["R_diag"][e, i]
            assert np.abs(L + L.conj().T).max() <= 1e-12 * np.abs(L).max()
            assert np.linalg.eigvalsh(-1j * L).min() >= -1e-9 * np.abs(L).max()
            assert np.linalg.eigvalsh(1j * G).min() >= -1e-9 * np.abs(G).max()
            A = 1j * (R - R.conj().T)
            assert np.linalg.eigvalsh(0.5 * (A + A.conj().T)).min() >= -1e-9 * np.abs(A).max()


@pytest.mark.gpu
def test_golden_gpu_matches_stored_values():
    from gpu_util import run_g
    s, d, blocks = load()
    res = run_g(s)
    assert (res["status"] == 0).all()
    for e in range(len(s.energies)):
        for k in KEYS:
            errs = block_errors(res[k][e], blocks[k][e], abs_floor=d["lesser_abs_floor"][e] if k[0] in "LG" else 0.0)
            tol = d["tol"][e][k]
            assert tol == TOL_FP64
            assert errs.max() <= tol, (k, e, errs.max(), tol)
