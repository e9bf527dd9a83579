"""The autotuner's knobs on the GPU: every combination of FP64 output tile and inversion panel
width solves to the oracle's tolerance (b = 130: blocked inversions, ragged tiles), and the tuner
picks a configuration by coordinate descent and caches it."""
import numpy as np
import pytest

import synthetic
from gpu_util import compare_g, run_g

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tile,panel", [(16, 0), (32, 0), (32, 8), (16, 4)])
def test_kernel_shape_knobs_keep_parity(tile, panel):
    import torch
    from paper_2508_19138_gb300.highlevel import GSolver
    s = synthetic.random_device(130, 3, 130, 3)
    solver = GSolver(s.nb, s.bs, 3, s.eta, s.kT, s.mu_left, s.mu_right, gemm_tile=tile, inv_panel=panel)
    solver.set_inputs(s.H_diag, s.H_upper)
    outs, status = solver.solve(s.energies)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    res = {w + "_" + k: getattr(o, k).cpu().numpy() for w, o in outs.items() for k in ("diag", "upper", "lower")
           if getattr(o, k) is not None}
    for e in range(3):
        _, bad = compare_g(res, s, e, e)
        assert not bad, (tile, panel, e, bad)
    solver.close()


def test_tuner_picks_and_caches(tmp_path):
    from paper_2508_19138_gb300 import autotune
    s = synthetic.random_device(9, 4, 96, 16)
    path = str(tmp_path / "tune.json")
    res = autotune.tune_g(s.nb, s.bs, s.H_diag, s.H_upper, s.energies, eta=s.eta, kT=s.kT, chunks=(4, 8),
                          tiles=(32, 16), panels=(0,), cache_path=path)
    assert not res["cached"]
    assert res["best"]["max_energies"] in (4, 8) and res["best"]["gemm_tile"] in (32, 16)
    again = autotune.tune_g(s.nb, s.bs, s.H_diag, s.H_upper, s.energies, eta=s.eta, kT=s.kT, cache_path=path)
    assert again["cached"] and again["best"] == res["best"]
