"""The error bound the split-GEMM tests use, checked against an exact model of the scheme.

The sliced product (Ozaki et al. 2012, error-free splitting) as the library describes it: each
row of op(A) and column of op(B) is scaled by R = 2^(E - 1022) (E its largest biased exponent),
rounded to X = round(|v| / R 2^(7S-1)) and written as S balanced base-128 digits; products of
digit pairs (s, t) with s + t <= S + 1 are summed exactly, weighted by 2^(-7(s + t - 2)) and
accumulated in fixed point with F = min(7S - 9, 50 - log2 K') fractional bits (pairs below the
resolution rounded to it).  This model, in exact integer arithmetic, stays within the bound
    |C - AB|_ij <= 2^(5 - 7S) k max_p |A_ip| max_p |B_pj|
of tests/test_gpu_split.py, and the bound is not loose by more than a small factor."""
import math

import numpy as np
import pytest


def row_exponents(A):
    """Largest biased IEEE exponent of each row (zeros count as exponent 1)."""
    e = np.frexp(np.abs(A))[1] + 1022              # biased exponent of |v| in [2^(e-1023), 2^(e-1022))
    e = np.where(A == 0, 1, e)
    return e.max(axis=1)


def digits(A, S):
    """Balanced base-128 digits [S, m, k] (int64) and scale exponents (R = 2^(E - 1022)) per row."""
    E = row_exponents(A)
    m, k = A.shape
    D = np.zeros((S, m, k), dtype=np.int64)
    for i in range(m):
        for p in range(k):
            v = A[i, p]
            X = int(round(math.ldexp(abs(v), 7 * S - 1 - (int(E[i]) - 1022))))   # exact: |v| has 53 bits
            sg = -1 if v < 0 else 1
            for s in range(S - 1, 0, -1):
                d = X & 127
                X >>= 7
                if d >= 64:
                    d -= 128
                    X += 1
                D[s, i, p] = sg * d
            D[0, i, p] = sg * X
    return D, E


def model_product(A, B, S):
    """The scheme's result for real A (m x k) and B (k x n)."""
    k = A.shape[1]
    Da, Ea = digits(A, S)
    Db, Eb = digits(B.T, S)                         # columns of B
    Kp = 2 * k                                      # the realified depth of a complex product
    F = min(7 * S - 9, 50 - int(math.ceil(math.log2(max(Kp, 2)))))
    acc = np.zeros((A.shape[0], B.shape[1]), dtype=object)
    for s in range(1, S + 1):
        for t in range(1, S + 2 - s):
            P = (Da[s - 1] @ Db[t - 1].T).astype(object)      # exact: |d_s d_t| <= 2^12, k small
            e = F - 7 * (s + t - 2)
            if e >= 0:
                acc += P * (1 << e)
            else:                                             # rounded to the resolution 2^-F
                acc += np.vectorize(lambda x: int(round(x / (1 << -e))))(P)
    out = np.zeros(acc.shape)
    for i in range(acc.shape[0]):
        for j in range(acc.shape[1]):
            out[i, j] = math.ldexp(float(acc[i, j]), int(Ea[i]) + int(Eb[j]) - 2044 - 12 - F)
    return out


@pytest.mark.parametrize("S", [3, 4, 6])
@pytest.mark.parametrize("k", [5, 40])
def test_scheme_within_the_test_bound(S, k):
    rng = np.random.default_rng(10 * S + k)
    m, n = 6, 5
    A = rng.standard_normal((m, k)) * np.exp(rng.uniform(-6, 6, (m, k)))   # wide range inside rows
    B = rng.standard_normal((k, n))
    got = model_product(A, B, S)
    ref = A @ B
    bound = 2.0 ** (5 - 7 * S) * k * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :]
    bound = bound + 1e-15 * (np.abs(A) @ np.abs(B))
    ratio = (np.abs(got - ref) / bound).max()
    assert ratio <= 1.0
    if S <= 4:      # at 6 slices the scheme's error is at the FP64 rounding of the reference
        assert ratio > 2.0 ** -12


def test_dropping_the_pair_truncation_is_seen():
    """Keeping every pair (s, t) would be more accurate; the s + t <= S + 1 truncation is what the
    bound accounts for: with 3 slices the truncated model's error is well above the full model's."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((4, 30))
    B = rng.standard_normal((30, 4))
    err3 = np.abs(model_product(A, B, 3) - A @ B).max()
    err5 = np.abs(model_product(A, B, 5) - A @ B).max()
    assert err3 > 100 * err5
