"""Bounded device waits driven to expiry (failure detection without a GPU fault).

The tensor-core GEMM's pipeline waits on shared-memory barriers are bounded.  The test hook
bt_debug_split_stall makes the MMA warp wait on a barrier that nothing completes, with a short
limit: every CTA then records BT_ERR_TIMEOUT, stops issuing, waits for the copies and products it
already issued, frees its tensor memory and exits.  The solve reports BT_ERR_TIMEOUT for every
energy of the chunk through the C ABI, and the next solve on the same context (hook off) is
correct against the oracle: its kernels allocate the tensor memory again, which they could not
if the timed-out CTAs had kept it."""
import numpy as np
import pytest

import synthetic
from gpu_util import TOL_SPLIT, compare_g

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scope", [0, 1])
def test_split_timeout_reported_then_context_recovers(scope):
    import torch
    import paper_2508_19138_gb300 as pkg
    from paper_2508_19138_gb300.highlevel import GSolver
    s = synthetic.random_device(71, 3, 64, 2)
    solver = GSolver(s.nb, s.bs, 2, s.eta, s.kT, s.mu_left, s.mu_right, obc=True, precision=pkg.BT_SPLIT,
                     split_scope=scope)
    solver.set_inputs(s.H_diag, s.H_upper)
    outs, status = solver.allocate_outputs(2)
    try:
        pkg.bt_debug_split_stall(20_000_000, -1)  # 20 ms on a barrier nothing completes
        solver.solve(s.energies, outs, status)
        torch.cuda.synchronize()
    finally:
        pkg.bt_debug_split_stall(0, 0)
    assert status.cpu().numpy().tolist() == [pkg.BT_ERR_TIMEOUT] * 2
    solver.solve(s.energies, outs, status)
    torch.cuda.synchronize()
    assert status.cpu().numpy().tolist() == [0, 0]
    res = {}
    for w, o in outs.items():
        res[w + "_diag"] = o.diag.cpu().numpy()
        res[w + "_upper"] = o.upper.cpu().numpy()
        if o.lower is not None:
            res[w + "_lower"] = o.lower.cpu().numpy()
    for e in range(2):
        _, bad = compare_g(res, s, e, e, tol=TOL_SPLIT)
        assert not bad, (e, bad)
    solver.close()
