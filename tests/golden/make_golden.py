"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

random_3x4.json: selected blocks of G^R, G^<, G^> (Sec. 3, Eq. 1 and Table 2: dense inverse of
M~ = E + i eta - H - B^R_OBC and X^<> = X^R B^<> X^R^H, symmetrised as in Sec. 5.2) for a seeded
3-block device of block size 4 with the lead surface functions of Eq. 4 from the direct route of
Eq. 6 (oracle.surface_gf_eig), at three energies inside the lead bands.  Regenerate with `python tests/golden/make_golden.py`; a change of the
stored numbers must name, in its commit message, the passage of the paper that justifies it.

w16x1024_e64.npz (`python tests/golden/make_golden.py w`, about 15 minutes on 8 cores): the W
system of 16 cells of 1024 atoms at energy index 64, from oracle.solve_w_sampled (Table 2, right
column: rows of X^R = (I - V P^R)^{-1} by banded LU, W^R = X^R V, W^<> = X^R V P^<> V^H X^R^H,
symmetrised as in Sec. 5.2) for block rows 0, 7 and 15: per block its Frobenius norm and the
values at W_SAMPLES entries drawn from a seeded generator (the indices are regenerated from the
seed by the test, so only values are stored).
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


W_ENERGY = 64
W_BLOCKS = (0, 7, 15)
W_SAMPLES = 512
W_KEYS = ("R_diag", "R_upper", "R_lower", "L_diag", "L_upper", "G_diag", "G_upper")


def w_sample_indices(bs, block, key):
    """Flat indices of the sampled entries of one block (seeded; shared with the test)."""
    rng = np.random.default_rng(90000 + 16 * block + W_KEYS.index(key))
    return rng.choice(bs * bs, size=W_SAMPLES, replace=False)


def main_w():
    ws = synthetic.w_system_16x1024()
    ref = oracle.solve_w_sampled(ws, W_ENERGY, list(W_BLOCKS))
    names, fro, vals = [], [], []
    for i in W_BLOCKS:
        for k in W_KEYS:
            if k not in ref[i]:
                continue
            blk = ref[i][k]
            names.append(f"{i}:{k}")
            fro.append(np.linalg.norm(blk))
            vals.append(blk.reshape(-1)[w_sample_indices(ws.bs, i, k)])
    np.savez_compressed(os.path.join(HERE, "w16x1024_e64.npz"), names=np.array(names), fro=np.array(fro),
                        vals=np.array(vals), energy=np.array(W_ENERGY))


def main():
    sys.path.insert(0, os.path.dirname(HERE))
    from gpu_util import TOL_FP64, lesser_floor  # oracle-only helpers of the tests
    s = system()
    out = {"case": CASE, "source": "oracle.solve_g (dense inverse, Sec. 3 Eq. 1, Table 2; symmetrised, Sec. 5.2; "
                                   "lead surface functions by the direct route of Eq. 6)",
           "energies": s.energies.tolist(), "blocks": {k: [] for k in KEYS},
           # per energy: absolute floor of the lesser/greater comparisons (FP64 rounding of the
           # boundary broadening) and the per-output tolerance (the FP64 tolerance)
           "lesser_abs_floor": [], "tol": []}
    for e in range(len(s.energies)):
        ref = oracle.solve_g(s, e, surface="eig")
        for k in KEYS:
            out["blocks"][k].append(to_pairs(ref[k]))
        out["lesser_abs_floor"].append(0.01 * lesser_floor(ref))
        out["tol"].append({k: TOL_FP64 for k in KEYS})
    with open(os.path.join(HERE, "random_3x4.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))
        f.write("\n")


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "w":
        main_w()
    else:
        main()
