"""The readings of the paper that the CUDA sweep relies on, checked on the CPU: a plain numpy
RGF (Sec. 4.3.2, Eq. 9-12, written here from the equations with the readings applied) against the
dense oracle, and each reading against its alternative.

* R1: y_i of Eq. 10 with x^R_{i-1} (the printed x^<>_{i-1} disagrees with the dense inverse);
* R3: the off-diagonal lesser block X^<>_{i,i+1};
* R15: Z_i of Eq. 12 equals U1 D^H with D the first term of X^<>_{i,i+1}, when x^<>_i is
  exactly anti-Hermitian;
* Sec. 5.2 symmetry enforced inside the sweep: every sandwich made exactly anti-Hermitian,
  element by element, matches the dense result; mirroring whole 32-wide tiles does not."""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import block_errors, lesser_floor


def _blocks(A, i, j, bs):
    return A[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs]


def antiherm_elementwise(C):
    U = np.triu(C, 1)
    return U - U.conj().T + np.diag(1j * np.diag(C).imag)


def antiherm_tiles(C, tile=32):
    """Tiles on and above the diagonal kept, tiles below replaced by the mirror image."""
    out = C.copy()
    n = C.shape[0]
    for r in range(n):
        for c in range(n):
            if r // tile > c // tile:
                out[r, c] = -np.conj(C[c, r])
    return out


def rgf(M, B, nb, bs, y_with_lesser=False, z_from_d=False, sandwich=None):
    """Selected blocks of X^R and X^< by the forward (Eq. 9-10) and backward (Eq. 11-12) passes;
    B may have off-diagonal blocks.  sandwich(C) post-processes every x B x^H product."""
    S = sandwich or (lambda C: C)
    blk = lambda A, i, j: _blocks(A, i, j, bs)
    xR, xL = [None] * nb, [None] * nb
    for i in range(nb):
        Mi = blk(M, i, i).copy()
        Bi = blk(B, i, i).copy()
        if i > 0:
            Mi -= blk(M, i, i - 1) @ xR[i - 1] @ blk(M, i - 1, i)
            Bi = S(Bi + blk(M, i, i - 1) @ xL[i - 1] @ blk(M, i, i - 1).conj().T)
            prev = xL[i - 1] if y_with_lesser else xR[i - 1]
            y = blk(M, i, i - 1) @ prev @ blk(B, i - 1, i)
            Bi = Bi - (y - y.conj().T)
        xR[i] = np.linalg.inv(Mi)
        xL[i] = S(xR[i] @ Bi @ xR[i].conj().T)
    XR, XL = xR[:], xL[:]
    XRu, XLu = [None] * (nb - 1), [None] * (nb - 1)
    for i in range(nb - 2, -1, -1):
        U1 = xR[i] @ blk(M, i, i + 1)
        W1 = blk(M, i + 1, i) @ xR[i]
        XRu[i] = -U1 @ XR[i + 1]
        V1 = XR[i + 1] @ blk(M, i + 1, i)
        D = -xL[i] @ V1.conj().T
        XLu[i] = D - U1 @ XL[i + 1] + xR[i] @ blk(B, i, i + 1) @ XR[i + 1].conj().T
        Z = U1 @ D.conj().T if z_from_d else -XRu[i] @ blk(M, i + 1, i) @ xL[i]
        Yb = -(xR[i] @ blk(B, i, i + 1)) @ XRu[i].conj().T
        XL[i] = S(xL[i] + U1 @ XL[i + 1] @ U1.conj().T) + (Z - Z.conj().T) - (Yb - Yb.conj().T)
        XR[i] = xR[i] - XRu[i] @ W1
    return np.array(XR), np.array(XL), np.array(XRu), np.array(XLu)


def check(s, e, **kw):
    ref = oracle.solve_g(s, e, symmetrize=False)
    M, BL = ref["M"], ref["BL"]
    XR, XL, XRu, XLu = rgf(M, BL, s.nb, s.bs, **kw)
    fl = 0.01 * lesser_floor(ref)
    sym = 0.5 * (XL - np.conj(np.swapaxes(XL, 1, 2)))
    refsym = 0.5 * (ref["L_diag"] - np.conj(np.swapaxes(ref["L_diag"], 1, 2)))
    return (block_errors(XR, ref["R_diag"]).max(), block_errors(sym, refsym, abs_floor=fl).max(),
            block_errors(XLu, ref["L_upper"], abs_floor=fl).max(), block_errors(XRu, ref["R_upper"]).max())


def banded_lesser_system(seed, nb, bs):
    """A device whose lesser right-hand side has off-diagonal blocks (as in the W system): the
    dense oracle system with B^< replaced by an anti-Hermitian block-tridiagonal matrix."""
    s = synthetic.random_device(seed, nb, bs, 3)
    rng = np.random.default_rng(seed + 1)
    n = nb * bs
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    mask = np.zeros((n, n), bool)
    for i in range(nb):
        for j in range(max(0, i - 1), min(nb, i + 2)):
            mask[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = True
    A = np.where(mask, G @ G.conj().T / n, 0.0)  # Hermitian PSD-ish, block-tridiagonal
    return s, -1j * A


@pytest.mark.parametrize("seed,nb,bs", [(3, 4, 6), (5, 5, 5)])
def test_rgf_readings_match_dense(seed, nb, bs):
    s = synthetic.random_device(seed, nb, bs, 5)
    for e in range(5):
        errs = check(s, e)
        assert max(errs) < 1e-10, errs


@pytest.mark.parametrize("seed,nb,bs", [(7, 4, 5), (8, 3, 7)])
def test_r1_y_with_retarded_function(seed, nb, bs):
    """With an off-diagonal lesser right-hand side the y_i term matters: x^R_{i-1} (R1) matches the
    dense X^R B X^R^H, the printed x^<>_{i-1} does not."""
    s, BL = banded_lesser_system(seed, nb, bs)
    e = 1
    M = oracle.assemble_g(s, e)[0]
    XRd = np.linalg.inv(M)
    XLd = XRd @ BL @ XRd.conj().T
    ref_diag = np.array([_blocks(XLd, i, i, bs) for i in range(nb)])
    ref_up = np.array([_blocks(XLd, i, i + 1, bs) for i in range(nb - 1)])
    good = rgf(M, BL, nb, bs)
    bad = rgf(M, BL, nb, bs, y_with_lesser=True)
    assert block_errors(good[1], ref_diag).max() < 1e-10
    assert block_errors(good[3], ref_up).max() < 1e-10
    assert block_errors(bad[1], ref_diag).max() > 1e-3


@pytest.mark.parametrize("seed,nb,bs", [(11, 4, 6), (230, 4, 40)])
def test_r15_z_from_first_offdiagonal_term(seed, nb, bs):
    s = synthetic.random_device(seed, nb, bs, 5)
    for e in range(5):
        errs = check(s, e, z_from_d=True, sandwich=antiherm_elementwise)
        assert max(errs) < 1e-10, (e, errs)


def test_symmetry_inside_sweep_elementwise_not_tiles():
    """Exactly anti-Hermitian sandwiches (element by element) keep the dense accuracy on a 4 x 130
    device; mirroring whole 32-wide tiles turns the operands' Hermitian rounding noise into
    anti-Hermitian error far above it."""
    s = synthetic.random_device(230, 4, 130, 5)
    e = 2
    good = check(s, e, sandwich=antiherm_elementwise)
    tiles = check(s, e, sandwich=antiherm_tiles)
    assert good[1] < 1e-12
    assert tiles[1] > 100 * good[1]
