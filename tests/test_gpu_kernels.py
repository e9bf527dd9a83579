"""GPU unit tests of the building blocks through the C ABI: complex FP64 GEMM, batched
Gauss-Jordan inverse, Sancho-Rubio decimation, each against numpy / the CPU oracle."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    import paper_2508_19138_gb300 as p
    assert torch.cuda.is_available()
    p.library()
    return p


def cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("m,n,k", [(32, 32, 32), (33, 17, 70), (416, 416, 416), (1, 5, 3), (100, 64, 1)])
@pytest.mark.parametrize("opA,opB", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_zgemm_matches_numpy(pkg, m, n, k, opA, opB):
    import torch
    rng = np.random.default_rng(m * 7 + n + k)
    batch = 3
    A = cplx(rng, (batch, m, k) if opA == 0 else (batch, k, m))
    B = cplx(rng, (batch, k, n) if opB == 0 else (batch, n, k))
    C0 = cplx(rng, (batch, m, n))
    alpha, beta = 0.7 - 0.2j, -0.5 + 1.5j
    opa = A if opA == 0 else np.conj(np.swapaxes(A, 1, 2))
    opb = B if opB == 0 else np.conj(np.swapaxes(B, 1, 2))
    ref = alpha * opa @ opb + beta * C0
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C0))
    pkg.bt_zgemm_batched(m, n, k, alpha, dA, A.shape[2], A.shape[1] * A.shape[2], opA, dB, B.shape[2],
                         B.shape[1] * B.shape[2], opB, beta, dC, n, m * n, batch)
    got = dC.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max()) * np.sqrt(k)


def test_zgemm_shared_operand_and_beta_zero(pkg):
    import torch
    rng = np.random.default_rng(9)
    A = cplx(rng, (40, 40))
    B = cplx(rng, (5, 40, 40))
    ref = A[None] @ B
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full((5, 40, 40), float("nan"), dtype=torch.complex128, device="cuda")  # beta=0 must not read C
    pkg.bt_zgemm_batched(40, 40, 40, 1.0, dA, 40, 0, 0, dB, 40, 1600, 0, 0.0, dC, 40, 1600, 5)
    assert np.abs(dC.cpu().numpy() - ref).max() < 1e-12


@pytest.mark.parametrize("n", [1, 7, 32, 33, 96, 97, 130, 416])
def test_zinv_matches_numpy(pkg, n):
    import torch
    rng = np.random.default_rng(n)
    batch = 4
    A = cplx(rng, (batch, n, n))
    A[1] += 3 * np.eye(n)
    A[2] = A[2] * 1e-3  # scaled
    ref = np.linalg.inv(A)
    dA = torch.from_numpy(A).cuda()
    info = torch.zeros(batch, dtype=torch.int32, device="cuda")
    pkg.bt_zinv_batched(n, dA, n * n, batch, info)
    assert info.cpu().numpy().tolist() == [0] * batch
    got = dA.cpu().numpy()
    for b in range(batch):
        cond = np.linalg.cond(A[b])
        assert np.linalg.norm(got[b] - ref[b]) / np.linalg.norm(ref[b]) < 1e-15 * cond * n


def test_zinv_pivoting_needed(pkg):
    """A matrix with a zero leading entry needs the row exchange."""
    import torch
    A = np.array([[0, 1, 2], [1, 0, 3], [4, -3, 8]], dtype=np.complex128)
    dA = torch.from_numpy(A[None].copy()).cuda()
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    pkg.bt_zinv_batched(3, dA, 9, 1, info)
    assert int(info[0]) == 0
    assert np.abs(dA.cpu().numpy()[0] - np.linalg.inv(A)).max() < 1e-14


@pytest.mark.parametrize("n", [200, 416])
def test_zinv_far_pivots(pkg, n):
    """Pivots in rows owned by other CTAs of the panel cluster: a matrix dominated by its
    anti-diagonal (every pivot comes from the far end), plus ties of equal magnitude."""
    import torch
    rng = np.random.default_rng(n + 5)
    A = np.zeros((3, n, n), dtype=np.complex128)
    J = np.fliplr(np.eye(n))
    A[0] = 4.0 * J + 0.1 * cplx(rng, (n, n))
    A[1] = J * (1.0 + 1.0j) + 0.05 * cplx(rng, (n, n))
    A[2] = np.where(rng.random((n, n)) < 0.5, 1.0, -1.0) + 0.0j  # many exact ties in |re| + |im|
    A[2] += 0.01 * n * np.eye(n)
    ref = np.linalg.inv(A)
    dA = torch.from_numpy(A).cuda()
    info = torch.zeros(3, dtype=torch.int32, device="cuda")
    pkg.bt_zinv_batched(n, dA, n * n, 3, info)
    assert info.cpu().numpy().tolist() == [0, 0, 0]
    got = dA.cpu().numpy()
    for b in range(3):
        cond = np.linalg.cond(A[b])
        assert np.linalg.norm(got[b] - ref[b]) / np.linalg.norm(ref[b]) < 1e-15 * cond * n


@pytest.mark.parametrize("n", [4, 130, 416])
def test_zinv_reports_singular_and_nonfinite(pkg, n):
    import torch
    rng = np.random.default_rng(1)
    A = cplx(rng, (3, n, n))
    A[0, :, 1] = 0.0          # singular: a zero column
    A[2, 0, 0] = np.nan       # non-finite
    dA = torch.from_numpy(A).cuda()
    info = torch.zeros(3, dtype=torch.int32, device="cuda")
    pkg.bt_zinv_batched(n, dA, n * n, 3, info)
    got = info.cpu().numpy().tolist()
    assert got[0] == pkg.BT_ERR_SINGULAR
    assert got[1] == 0
    assert got[2] == pkg.BT_ERR_NONFINITE


@pytest.mark.parametrize("bs", [1, 8, 33, 130])
def test_decimation_matches_oracle(pkg, bs):
    import torch
    rng = np.random.default_rng(bs)
    batch = 3
    ms, ns, nps, refs, its = [], [], [], [], []
    for b in range(batch):
        h00 = cplx(rng, (bs, bs))
        h00 = (h00 + h00.conj().T) / 2 / np.sqrt(bs)
        h01 = 0.5 * cplx(rng, (bs, bs)) / np.sqrt(bs)
        z = (-0.5 + 0.5 * b) + 1e-4j
        m, n, n_ = z * np.eye(bs) - h00, -h01, -h01.conj().T
        _, it, ok = oracle.sancho_rubio(m, n, n_)
        assert ok
        # reference: the direct route (Eq. 6); at eta = 1e-4 plain FP64 decimation is accurate
        x = oracle.surface_gf_eig(m, n, n_)
        ms.append(m); ns.append(n); nps.append(n_); refs.append(x); its.append(it)
    dm, dn, dnp = (torch.from_numpy(np.ascontiguousarray(np.stack(a))).cuda() for a in (ms, ns, nps))
    x = torch.empty_like(dm)
    sig = torch.empty_like(dm)
    iters = torch.zeros(batch, dtype=torch.int32, device="cuda")
    info = torch.zeros(batch, dtype=torch.int32, device="cuda")
    pkg.bt_decimate_batched(bs, batch, dm, dn, dnp, 1e-14, 100, x, sig, iters, info)
    assert info.cpu().numpy().tolist() == [0] * batch
    got = x.cpu().numpy()
    gi = iters.cpu().numpy()
    for b in range(batch):
        tol = 1e-10
        assert np.linalg.norm(got[b] - refs[b]) / np.linalg.norm(refs[b]) < tol
        assert abs(int(gi[b]) - its[b]) <= 1
        sref = ns[b] @ refs[b] @ nps[b]
        assert np.linalg.norm(sig.cpu().numpy()[b] - sref) / np.linalg.norm(sref) < tol


def test_decimation_iteration_cap_reports_not_converged(pkg):
    import torch
    bs = 4
    rng = np.random.default_rng(3)
    h00 = cplx(rng, (bs, bs))
    h00 = (h00 + h00.conj().T) / 2
    m = (0.1 + 1e-9j) * np.eye(bs) - h00
    n = -np.eye(bs, dtype=np.complex128)
    dm, dn = (torch.from_numpy(np.ascontiguousarray(m[None])).cuda(),
              torch.from_numpy(np.ascontiguousarray(n[None])).cuda())
    x = torch.empty_like(dm)
    iters = torch.zeros(1, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    pkg.bt_decimate_batched(bs, 1, dm, dn, dn, 1e-14, 2, x, None, iters, info)
    assert int(info[0]) == pkg.BT_ERR_NOT_CONVERGED
    assert int(iters[0]) == 2
