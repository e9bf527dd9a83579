"""Energy convolution by FFT (Sec. 4.4, Eq. 3) on the GPU against the oracle's explicit sum,
element by element: per element series the relative Frobenius error over the written window
must be <= 1e-10 (the FP64 tolerance), at transform lengths from 2 to 4096, ragged element
counts (tiles of several series), strided energy-major layouts, output windows, the reversed and
conjugated second series, and the layout of the solver's outputs (G^< diagonal blocks)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

TOL = 1e-10


def cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def run(a, b, n_elem, lda, ldb, scale, m0, n_out, flags, ldc=None):
    import torch
    import paper_2508_19138_gb300 as pkg
    ldc = ldc or n_elem
    A = torch.from_numpy(a.reshape(-1)).cuda()
    B = torch.from_numpy(b.reshape(-1)).cuda()
    C = torch.full((n_out * ldc,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
    pkg.bt_energy_convolve(n_elem, a.shape[0], b.shape[0], A, lda, B, ldb, C, ldc, scale=scale, m0=m0,
                           n_out=n_out, flags=flags)
    torch.cuda.synchronize()
    return C.cpu().numpy().reshape(n_out, ldc)


def series_errors(got, want):
    num = np.linalg.norm(got - want, axis=0)
    den = np.linalg.norm(want, axis=0)
    return num / np.maximum(den, 1e-300)


@pytest.mark.parametrize("na,nb,n_elem,pad", [(512, 512, 301, 0), (7, 3, 1000, 5), (1, 1, 33, 0),
                                              (2048, 2049, 3, 1), (100, 300, 64, 13), (513, 512, 17, 0)])
@pytest.mark.parametrize("flags", [0, 1, 2, 3])
def test_convolution_matches_oracle(na, nb, n_elem, pad, flags):
    import paper_2508_19138_gb300 as pkg
    rng = np.random.default_rng(na * 7 + nb + flags)
    lda = ldb = n_elem + pad
    a = cplx(rng, (na, lda))
    b = cplx(rng, (nb, ldb))
    full = na + nb - 1
    m0 = full // 5
    n_out = full - m0 - full // 7
    s = 0.37 - 1.3j
    got = run(a, b, n_elem, lda, ldb, s, m0, n_out, flags)
    want = oracle.energy_convolve(a[:, :n_elem], b[:, :n_elem], scale=s, m0=m0, n_out=n_out,
                                  reverse_b=bool(flags & pkg.BT_CONV_REVERSE_B), conj_b=bool(flags & pkg.BT_CONV_CONJ_B))
    err = series_errors(got[:, :n_elem], want)
    assert err.max() <= TOL, err.max()


def test_convolution_of_solver_outputs_layout():
    """The polarization-like product of two G^< diagonal-block series straight from the solver's
    [E][nb][bs][bs] output layout (lda = nb bs^2), 64 energies, against the oracle on the same
    arrays; and the packed upper-triangle layout gives the same entries."""
    import torch
    import paper_2508_19138_gb300 as pkg
    from gpu_util import unpack_upper
    import synthetic
    from paper_2508_19138_gb300.highlevel import GSolver
    s = synthetic.random_device(5, 3, 16, 64)
    solver = GSolver(s.nb, s.bs, 64, s.eta, s.kT, s.mu_left, s.mu_right)
    solver.set_inputs(s.H_diag, s.H_upper)
    full_outs, st1 = solver.allocate_outputs(64)
    packed, st2 = solver.allocate_outputs(64, packed_lg=True)
    solver.solve(s.energies, full_outs, st1)
    solver.solve(s.energies, packed, st2)
    torch.cuda.synchronize()
    GL, GG = full_outs["L"].diag, full_outs["G"].diag
    n_elem = s.nb * s.bs * s.bs
    C = torch.empty((127, n_elem), dtype=torch.complex128, device="cuda")
    pkg.bt_energy_convolve(n_elem, 64, 64, GL, n_elem, GG, n_elem, C, n_elem, scale=0.01j,
                           flags=pkg.BT_CONV_REVERSE_B)
    P = torch.empty((127, s.nb * s.bs * (s.bs + 1) // 2), dtype=torch.complex128, device="cuda")
    npk = P.shape[1]
    pkg.bt_energy_convolve(npk, 64, 64, packed["L"].diag, npk, packed["G"].diag, npk, P, npk, scale=0.01j,
                           flags=pkg.BT_CONV_REVERSE_B)
    torch.cuda.synchronize()
    gl = GL.cpu().numpy().reshape(64, -1)
    gg = GG.cpu().numpy().reshape(64, -1)
    want = oracle.energy_convolve(gl, gg, scale=0.01j, reverse_b=True)
    got = C.cpu().numpy()
    assert series_errors(got, want).max() <= TOL
    # packed: upper-triangle entries equal the full layout's
    iu = np.triu_indices(s.bs)
    full_u = got.reshape(127, s.nb, s.bs, s.bs)[:, :, iu[0], iu[1]]
    assert np.allclose(P.cpu().numpy().reshape(127, s.nb, -1), full_u, rtol=0, atol=1e-12 * np.abs(got).max())
    solver.close()


def test_rejects_bad_arguments():
    import torch
    import paper_2508_19138_gb300 as pkg
    A = torch.zeros(16, dtype=torch.complex128, device="cuda")
    with pytest.raises(pkg.BTError) as ei:
        pkg.bt_energy_convolve(4, 3000, 3000, A, 4, A, 4, A, 4)  # L = 8192 > 4096
    assert ei.value.status == pkg.BT_ERR_UNSUPPORTED
    with pytest.raises(pkg.BTError) as ei:
        pkg.bt_energy_convolve(4, 2, 2, A, 3, A, 4, A, 4)        # lda < n_elem
    assert ei.value.status == pkg.BT_ERR_INVALID_ARG
    with pytest.raises(pkg.BTError) as ei:
        pkg.bt_energy_convolve(4, 2, 2, A, 4, A, 4, A, 4, m0=2, n_out=2)  # window beyond na + nb - 1
    assert ei.value.status == pkg.BT_ERR_INVALID_ARG
