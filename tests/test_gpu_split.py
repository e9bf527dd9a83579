"""Split-precision (sliced bf16 on tcgen05) complex GEMM through the C ABI, against numpy
complex128 products: the error is bounded relative to |op(A)| |op(B)| (the Ozaki-scheme bound),
for ragged shapes, both operand orientations, complex alpha / beta and k beyond one K chunk."""
import numpy as np
import pytest

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


# Ozaki-scheme bound: every operand entry is truncated at 2^-7S of its row (op(A)) / column
# (op(B)) maximum and pairs with s + t > S + 1 are dropped, so
#     |C - AB|_ij <= c_S * k * max_p |op(A)_ip| * max_p |op(B)_pj|,  c_S = 2^(5 - 7S)
# (complex components and the dropped pairs folded into 2^5); FP64 rounding of the result adds
# a few ulps of |A||B|.
def scale(opa, opb):
    ra = np.maximum(np.abs(opa.real), np.abs(opa.imag)).max(axis=-1)        # [batch, m]
    cb = np.maximum(np.abs(opb.real), np.abs(opb.imag)).max(axis=-2)        # [batch, n]
    k = opa.shape[-1]
    return k * ra[..., :, None] * cb[..., None, :]


def within(got, ref, opa, opb, S, extra=0.0):
    lim = 2.0 ** (5 - 7 * S) * scale(opa, opb) + 1e-15 * (np.abs(opa) @ np.abs(opb)) + extra
    return np.all(np.abs(got - ref) <= lim), float((np.abs(got - ref) / lim).max())


@pytest.mark.parametrize("m,n,k", [(128, 64, 64), (416, 416, 416), (33, 17, 70), (1, 5, 3), (100, 130, 600)])
@pytest.mark.parametrize("opA,opB", [(0, 0), (1, 1), (0, 1), (1, 0)])
def test_split_zgemm_matches_numpy(pkg, m, n, k, opA, opB):
    import torch
    rng = np.random.default_rng(m + 3 * n + 7 * k + opA + 2 * opB)
    batch = 2
    A = cplx(rng, (batch, m, k) if opA == 0 else (batch, k, m))
    B = cplx(rng, (batch, k, n) if opB == 0 else (batch, n, k))
    A[0] *= np.exp(rng.uniform(-8, 8, size=A.shape[1:]))  # wide dynamic range inside rows / columns
    opa = A if opA == 0 else np.conj(np.swapaxes(A, 1, 2))
    opb = B if opB == 0 else np.conj(np.swapaxes(B, 1, 2))
    ref = opa @ opb
    mag = np.abs(opa) @ np.abs(opb)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.full((batch, m, n), float("nan"), dtype=torch.complex128, device="cuda")
    S = 6
    pkg.bt_split_zgemm_batched(m, n, k, 1.0, dA, A.shape[2], A.shape[1] * A.shape[2], opA, dB, B.shape[2],
                               B.shape[1] * B.shape[2], opB, 0.0, dC, n, m * n, batch, S)
    got = dC.cpu().numpy()
    assert np.isfinite(got).all()
    ok, worst = within(got, ref, opa, opb, S)
    assert ok, worst


@pytest.mark.parametrize("S", [4, 5, 6, 7, 8])
def test_split_error_decreases_with_slices(pkg, S):
    import torch
    rng = np.random.default_rng(11)
    m = n = k = 96
    A, B = cplx(rng, (1, m, k)), cplx(rng, (1, k, n))
    ref = A @ B
    mag = np.abs(A) @ np.abs(B)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros((1, m, n), dtype=torch.complex128, device="cuda")
    pkg.bt_split_zgemm_batched(m, n, k, 1.0, dA, k, m * k, 0, dB, n, k * n, 0, 0.0, dC, n, m * n, 1, S)
    ok, worst = within(dC.cpu().numpy(), ref, A, B, S)
    assert ok, worst


def test_split_alpha_beta_complex_and_shared_operand(pkg):
    import torch
    rng = np.random.default_rng(5)
    m, n, k, batch = 64, 48, 80, 3
    A = cplx(rng, (m, k))            # shared by every batch entry (stride 0)
    B = cplx(rng, (batch, k, n))
    C0 = cplx(rng, (batch, m, n))
    alpha, beta = 0.3 - 1.1j, -0.7 + 0.25j
    ref = alpha * (A[None] @ B) + beta * C0
    mag = np.abs(alpha) * (np.abs(A)[None] @ np.abs(B)) + np.abs(beta) * np.abs(C0)
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C0))
    pkg.bt_split_zgemm_batched(m, n, k, alpha, dA, k, 0, 0, dB, n, k * n, 0, beta, dC, n, m * n, batch, 6)
    ok, worst = within(dC.cpu().numpy(), ref, np.broadcast_to(A, (batch, m, k)) * abs(alpha), B, 6,
                       extra=1e-15 * np.abs(beta) * np.abs(C0))
    assert ok, worst


def test_split_long_k_accumulates_chunks(pkg):
    """k = 1100 > 512: three K chunks accumulated into C."""
    import torch
    rng = np.random.default_rng(7)
    m, n, k = 40, 24, 1100
    A, B = cplx(rng, (1, m, k)), cplx(rng, (1, k, n))
    C0 = cplx(rng, (1, m, n))
    ref = -1.0 * (A @ B) + 1.0 * C0
    mag = np.abs(A) @ np.abs(B) + np.abs(C0)
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C0))
    pkg.bt_split_zgemm_batched(m, n, k, -1.0, dA, k, m * k, 0, dB, n, k * n, 0, 1.0, dC, n, m * n, 1, 6)
    ok, worst = within(dC.cpu().numpy(), ref, A, B, 6, extra=1e-15 * np.abs(C0))
    assert ok, worst


def test_split_zero_and_tiny_rows(pkg):
    import torch
    rng = np.random.default_rng(9)
    m, n, k = 50, 40, 30
    A, B = cplx(rng, (1, m, k)), cplx(rng, (1, k, n))
    A[0, 3] = 0.0
    A[0, 7] *= 1e-200
    B[0, :, 5] *= 1e150
    ref = A @ B
    mag = np.abs(A) @ np.abs(B)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    dC = torch.zeros((1, m, n), dtype=torch.complex128, device="cuda")
    pkg.bt_split_zgemm_batched(m, n, k, 1.0, dA, k, m * k, 0, dB, n, k * n, 0, 0.0, dC, n, m * n, 1, 6)
    got = dC.cpu().numpy()
    assert np.all(got[0, 3] == 0)
    ok, worst = within(got, ref, A, B, 6)
    assert ok, worst
