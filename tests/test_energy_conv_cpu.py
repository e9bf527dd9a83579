"""Pins of the oracle's element-wise energy convolution (Sec. 4.4, Eq. 3): each against something
other than the oracle itself."""
import numpy as np
import pytest

import oracle


def cplx(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_delta_series_gives_a_shifted_copy():
    """b = delta at k0: c[m] = s a[m - k0] exactly."""
    rng = np.random.default_rng(1)
    a = cplx(rng, (17, 5))
    b = np.zeros((9, 5), complex)
    b[4] = 1.0
    c = oracle.energy_convolve(a, b, scale=0.5 - 2j)
    assert c.shape == (25, 5)
    want = np.zeros_like(c)
    want[4:4 + 17] = (0.5 - 2j) * a
    assert np.array_equal(c, want)


def test_geometric_series_closed_form():
    """a[k] = alpha^k, b[k] = beta^k: c[m] = sum_{k=lo}^{hi} alpha^(m-k) beta^k
    = alpha^m (r^lo - r^(hi+1)) / (1 - r), r = beta / alpha, lo = max(0, m - na + 1), hi = min(m, nb - 1)."""
    na, nb = 13, 7
    alpha = np.array([0.9 * np.exp(0.3j), -0.5 + 0.2j])
    beta = np.array([0.7 * np.exp(-1.1j), 0.3 - 0.6j])
    a = alpha[None, :] ** np.arange(na)[:, None]
    b = beta[None, :] ** np.arange(nb)[:, None]
    c = oracle.energy_convolve(a, b)
    r = beta / alpha
    for m in range(na + nb - 1):
        lo, hi = max(0, m - na + 1), min(m, nb - 1)
        want = alpha ** m * (r ** lo - r ** (hi + 1)) / (1 - r)
        assert np.allclose(c[m], want, rtol=1e-13, atol=1e-15)


def test_brute_force_plain_python_with_window_reverse_and_conjugate():
    rng = np.random.default_rng(3)
    na, nb = 6, 4
    a = cplx(rng, (na, 3))
    b = cplx(rng, (nb, 3))
    s = 1.5 + 0.25j
    for reverse in (False, True):
        for conj in (False, True):
            c = oracle.energy_convolve(a, b, scale=s, m0=2, n_out=5, reverse_b=reverse, conj_b=conj)
            for e in range(3):
                for mi, m in enumerate(range(2, 7)):
                    acc = 0j
                    for k in range(nb):
                        if 0 <= m - k < na:
                            bk = b[nb - 1 - k, e] if reverse else b[k, e]
                            acc += a[m - k, e] * (bk.conjugate() if conj else bk)
                    assert abs(c[mi, e] - s * acc) <= 1e-14 * max(1.0, abs(acc))


def test_commutative_and_matches_numpy_convolve():
    rng = np.random.default_rng(4)
    a = cplx(rng, (31, 2))
    b = cplx(rng, (31, 2))
    assert np.allclose(oracle.energy_convolve(a, b), oracle.energy_convolve(b, a), rtol=1e-14, atol=1e-13)
    for e in range(2):
        assert np.allclose(oracle.energy_convolve(a, b)[:, e], np.convolve(a[:, e], b[:, e]), rtol=1e-13, atol=1e-12)


def test_reversal_is_a_cross_correlation():
    """With b reversed, c[m] = sum_j a[j] b[j + nb - 1 - m]: the correlation of a and b."""
    rng = np.random.default_rng(5)
    a = cplx(rng, (8,))
    b = cplx(rng, (5,))
    c = oracle.energy_convolve(a, b, reverse_b=True)
    for m in range(12):
        want = sum(a[j] * b[j + 4 - m] for j in range(8) if 0 <= j + 4 - m < 5)
        assert abs(c[m] - want) <= 1e-13


@pytest.mark.parametrize("bad", ["shape"])
def test_rejects_mismatched_elements(bad):
    with pytest.raises(ValueError):
        oracle.energy_convolve(np.zeros((3, 2)), np.zeros((3, 4)))
