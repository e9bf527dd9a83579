"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

random_3x4.json: selected blocks of G^R, G^<, G^> (Sec. 3, Eq. 1 and Table 2: dense inverse of
M~ = E + i eta - H - B^R_OBC and X^<> = X^R B^<> X^R^H, symmetrised as in Sec. 5.2) for a seeded
3-block device of block size 4 with Sancho-Rubio contacts (Sec. 4.2, Eq. 4), at three energies
inside the lead bands.  Regenerate with `python tests/golden/make_golden.py`; a change of the
stored numbers must name, in its commit message, the passage of the paper that justifies it.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthetic  # noqa: E402

CASE = dict(seed=4242, nb=3, bs=4, n_energies=3, e_lo=-0.9, e_hi=0.6)
KEYS = ("R_diag", "R_upper", "R_lower", "L_diag", "L_upper", "G_diag", "G_upper")


def system():
    c = CASE
    return synthetic.random_device(c["seed"], c["nb"], c["bs"], c["n_energies"], e_lo=c["e_lo"], e_hi=c["e_hi"])


def to_pairs(a):
    a = np.asarray(a)
    return np.stack([a.real, a.imag], axis=-1).tolist()


def main():
    sys.path.insert(0, os.path.dirname(HERE))
    from gpu_util import TOL_FP64, lesser_floor, route_discrepancy  # oracle-only helpers of the tests
    s = system()
    out = {"case": CASE, "source": "oracle.solve_g (dense inverse, Sec. 3 Eq. 1, Table 2; symmetrised, Sec. 5.2)",
           "energies": s.energies.tolist(), "blocks": {k: [] for k in KEYS},
           # per energy: absolute floor of the lesser/greater comparisons and per-output tolerance,
           # both from the oracle (FP64 rounding of the boundary broadening; 10x the disagreement
           # of the oracle's two contact routes, never below the FP64 tolerance)
           "lesser_abs_floor": [], "tol": []}
    for e in range(len(s.energies)):
        ref = oracle.solve_g(s, e)
        for k in KEYS:
            out["blocks"][k].append(to_pairs(ref[k]))
        out["lesser_abs_floor"].append(0.01 * lesser_floor(ref))
        disc = route_discrepancy(s, e)
        out["tol"].append({k: max(TOL_FP64, 10.0 * disc.get(k, 0.0)) for k in KEYS})
    with open(os.path.join(HERE, "random_3x4.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    main()
