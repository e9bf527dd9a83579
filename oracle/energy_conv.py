"""Element-wise energy convolution (Sec. 4.4, Eq. 3) for the CPU oracle (test infrastructure only).

Eq. 3 gives the scattering self-energy (or the polarization) of an element (i, j) as an energy
integral of products of two particle descriptors, B_scatt(E) proportional to the integral of
X1(E - E') X2(E') over E'; each (i, j) entry is convolved independently of the others.  On a
uniform energy grid of spacing dE the integral becomes the discrete linear convolution

    c[m] = s * sum_k a[m - k] * b[k],   a[i] = 0 outside [0, na),  b[k] = 0 outside [0, nb),

with the proportionality constant and dE folded into the complex scale s, for 0 <= m < na + nb - 1.
Optional variants: the second series reversed in energy (b[k] -> b[nb - 1 - k], which turns the
convolution into a cross-correlation, the form of the polarization's E' - E argument) and / or
complex-conjugated (the transposed element of an anti-Hermitian quantity).

The oracle writes the definition out: an explicit sum over k, vectorised over the elements and
the output index only.  It is pinned by tests/test_energy_conv_cpu.py against a shifted copy
(delta series), the closed form of two geometric series, brute force in plain Python, the
reversal identity and numpy's own convolution.
"""
from __future__ import annotations

import numpy as np

__all__ = ["energy_convolve"]


def energy_convolve(a, b, scale=1.0, m0=0, n_out=None, reverse_b=False, conj_b=False):
    """Linear convolution of element series along axis 0 (Sec. 4.4, Eq. 3).

    a: [na, ...] and b: [nb, ...] with the same trailing (element) shape; returns
    c[m0 : m0 + n_out] of c[m] = scale * sum_k a[m - k] * b'[k], where b' is b, reversed in energy
    (reverse_b) and / or complex-conjugated (conj_b).  n_out defaults to na + nb - 1 - m0."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    na, nb = a.shape[0], b.shape[0]
    if a.shape[1:] != b.shape[1:]:
        raise ValueError("a and b must have the same element shape")
    if reverse_b:
        b = b[::-1]
    if conj_b:
        b = np.conj(b)
    full = na + nb - 1
    if n_out is None:
        n_out = full - m0
    c = np.zeros((full,) + a.shape[1:], dtype=np.complex128)
    for k in range(nb):
        # b[k] contributes a[i] b[k] to c[i + k]
        c[k:k + na] += a * b[k]
    return scale * c[m0:m0 + n_out]
