"""The tensor-core GEMM on CTA pairs (tcgen05 cta_group::2; pipeline stages of one or two K
blocks) against the one-CTA kernel.

Both compute every slice-pair product exactly in fp32 and sum them in the same uint64 fixed point,
so their results are bitwise equal, whatever the shape (an odd number of 128-row tiles pads the
last pair with zero rows), the operand forms and the coefficients.  The result is also checked
against the exact product (numpy, FP64) at the split path's accuracy; and a bounded wait of the
pair kernel driven to expiry is reported and leaves the context usable."""
import numpy as np
import pytest

import synthetic
from gpu_util import TOL_SPLIT, compare_g

pytestmark = pytest.mark.gpu

# (m, n, k, batch, opA, opB): 2n = 832 (7 tiles, last pair padded), 400 (4 tiles), 260 (3), 200 (2)
CASES = [(416, 416, 416, 3, 0, 0), (200, 200, 130, 4, 1, 0), (130, 130, 130, 2, 0, 1), (100, 100, 60, 3, 1, 1),
         (96, 208, 64, 2, 0, 0)]


def _run(pkg, torch, mode, m, n, k, batch, opA, opB, alpha, beta, A, B, C0):
    pkg.bt_debug_split_pair(mode)
    try:
        C = C0.clone()
        lda = k if opA == 0 else m
        ldb = n if opB == 0 else k
        pkg.bt_split_zgemm_batched(m, n, k, alpha, A, lda, A[0].numel(), opA, B, ldb, B[0].numel(), opB, beta, C, n,
                                   m * n, batch, 6)
        torch.cuda.synchronize()
    finally:
        pkg.bt_debug_split_pair(0)
    return C


@pytest.mark.parametrize("m,n,k,batch,opA,opB", CASES)
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-1.0, 1.0), (0.5 - 0.25j, 0.75j)])
def test_pair_bitwise_equals_single_cta(m, n, k, batch, opA, opB, alpha, beta):
    import torch
    import paper_2508_19138_gb300 as pkg
    g = torch.Generator(device="cuda").manual_seed(m * 7 + n * 3 + k + batch)
    shA = (batch, m, k) if opA == 0 else (batch, k, m)
    shB = (batch, k, n) if opB == 0 else (batch, n, k)
    A = torch.randn(shA, dtype=torch.complex128, device="cuda", generator=g)
    B = torch.randn(shB, dtype=torch.complex128, device="cuda", generator=g)
    C0 = torch.randn(batch, m, n, dtype=torch.complex128, device="cuda", generator=g)
    c1 = _run(pkg, torch, 1, m, n, k, batch, opA, opB, alpha, beta, A, B, C0)
    c2 = _run(pkg, torch, 2, m, n, k, batch, opA, opB, alpha, beta, A, B, C0)
    c3 = _run(pkg, torch, 3, m, n, k, batch, opA, opB, alpha, beta, A, B, C0)  # two K blocks per stage
    assert torch.equal(c1, c2), (c1 - c2).abs().max().item()
    assert torch.equal(c1, c3), (c1 - c3).abs().max().item()
    # against the exact product (FP64 on the host)
    a = A.cpu().numpy()
    b = B.cpu().numpy()
    opa = a if opA == 0 else np.conj(np.transpose(a, (0, 2, 1)))
    opb = b if opB == 0 else np.conj(np.transpose(b, (0, 2, 1)))
    ref = alpha * np.matmul(opa, opb) + beta * C0.cpu().numpy()
    got = c2.cpu().numpy()
    for i in range(batch):
        err = np.linalg.norm(got[i] - ref[i]) / np.linalg.norm(ref[i])
        assert err < 1e-11, (i, err)


@pytest.mark.parametrize("m,n,k,batch,opA,opB", CASES + [(416, 416, 416, 2, 0, 0), (256, 256, 1024, 2, 0, 1)])
def test_merged_accumulators_match_one_pair_per_accumulator(m, n, k, batch, opA, opB):
    """The default schedule (pairs of one weight class summed in one accumulator) against one pair
    per accumulator: the same exact products in the same fixed point, rounded at different points
    only for the classes below the fixed point's resolution, so the results agree far below the
    split path's error; both against the exact product."""
    import torch
    import paper_2508_19138_gb300 as pkg
    g = torch.Generator(device="cuda").manual_seed(m * 5 + n + k * 3 + batch)
    shA = (batch, m, k) if opA == 0 else (batch, k, m)
    shB = (batch, k, n) if opB == 0 else (batch, n, k)
    A = torch.randn(shA, dtype=torch.complex128, device="cuda", generator=g)
    B = torch.randn(shB, dtype=torch.complex128, device="cuda", generator=g)
    C0 = torch.randn(batch, m, n, dtype=torch.complex128, device="cuda", generator=g)
    got = {}
    for sched in (0, 1):
        pkg.bt_debug_split_sched(sched)
        try:
            got[sched] = _run(pkg, torch, 0, m, n, k, batch, opA, opB, 1.0, 0.0, A, B, C0)
        finally:
            pkg.bt_debug_split_sched(0)
    a = A.cpu().numpy()
    b = B.cpu().numpy()
    opa = a if opA == 0 else np.conj(np.transpose(a, (0, 2, 1)))
    opb = b if opB == 0 else np.conj(np.transpose(b, (0, 2, 1)))
    ref = np.matmul(opa, opb)
    g0, g1 = got[0].cpu().numpy(), got[1].cpu().numpy()
    for i in range(batch):
        nr = np.linalg.norm(ref[i])
        assert np.linalg.norm(g0[i] - g1[i]) / nr < 1e-12, i
        assert np.linalg.norm(g0[i] - ref[i]) / nr < 1e-11, i
        assert np.linalg.norm(g1[i] - ref[i]) / nr < 1e-11, i


def test_pair_timeout_reported_then_context_recovers():
    """b = 130: the products of the solve have 2n = 260 rows of C^T (three 128-row tiles) and run
    on CTA pairs; the stall hook makes the pair leader's MMA warp time out."""
    import torch
    import paper_2508_19138_gb300 as pkg
    from paper_2508_19138_gb300.highlevel import GSolver
    s = synthetic.random_device(73, 3, 130, 2)
    solver = GSolver(s.nb, s.bs, 2, s.eta, s.kT, s.mu_left, s.mu_right, obc=True, precision=pkg.BT_SPLIT,
                     split_scope=1)
    solver.set_inputs(s.H_diag, s.H_upper)
    outs, status = solver.allocate_outputs(2)
    pkg.bt_debug_split_pair(2)
    try:
        try:
            pkg.bt_debug_split_stall(20_000_000, -1)
            solver.solve(s.energies, outs, status)
            torch.cuda.synchronize()
        finally:
            pkg.bt_debug_split_stall(0, 0)
        assert status.cpu().numpy().tolist() == [pkg.BT_ERR_TIMEOUT] * 2
        solver.solve(s.energies, outs, status)
        torch.cuda.synchronize()
    finally:
        pkg.bt_debug_split_pair(0)
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
