"""Pins of the emulated-contraction oracle (oracle/emu.py), CPU only."""
import numpy as np
import pytest

from oracle import emu


def upper_mirrored(K):
    """the symmetric matrix with K's upper triangle (what the contraction returns)"""
    iu = np.triu_indices(K.shape[0])
    S = np.zeros_like(K)
    S[iu] = K[iu]
    S.T[iu] = K[iu]
    return S


def test_integer_operands_give_the_exact_product():
    rng = np.random.default_rng(0)
    A = rng.integers(-100, 101, (700, 9)).astype(float)
    B = rng.integers(-1000, 1001, (700, 9)).astype(float)
    want = upper_mirrored(A.T @ B)
    np.testing.assert_array_equal(emu.contract(A, B), want)
    np.testing.assert_array_equal(emu.contract(A, B, parts=1), want)


@pytest.mark.parametrize("seed", [0, 1])
def test_error_within_the_splitting_bound(seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(600, 7)) * 10.0 ** rng.uniform(-6, 6, (600, 7))
    B = rng.normal(size=(600, 7)) * 10.0 ** rng.uniform(-6, 6, (600, 7))
    K = emu.contract(A, B)
    exact = A.T @ B  # FP64 reference, itself within 600 eps |A|^T |B|
    ref_err = 600 * np.finfo(float).eps * (np.abs(A).T @ np.abs(B))
    iu = np.triu_indices(7)
    err = np.abs(K - exact)[iu]
    assert np.all(err <= 2.0 ** -50 * emu.error_bound(A, B)[iu] + ref_err[iu])


def test_level_sums_stay_exact_in_fp32():
    rng = np.random.default_rng(2)
    A = rng.uniform(-1, 1, (1024, 5))
    B = rng.uniform(-1, 1, (1024, 5))
    assert emu.level_bound(A, B) <= 2 ** 24


def test_slices_reconstruct_the_operand():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(512, 4)) * 1e3
    Q, e = emu.split(X)
    assert np.abs(Q).max() <= 64
    assert Q[1:].min() >= -64 and Q[1:].max() <= 63  # balanced digits after the first
    from fractions import Fraction
    for i in range(0, 512, 37):
        for j in range(4):
            rec = sum(Fraction(int(Q[t, i, j])) * Fraction(2) ** (-7 * (t + 1)) for t in range(emu.NS))
            rec *= Fraction(2) ** int(e[j])
            # the fixed-point rounding: at most 2^-57 of 2^e, and 2^e <= 4 max |x|
            assert abs(rec - Fraction(X[i, j])) <= Fraction(2) ** (int(e[j]) - 57)
    # a value whose bits end above 2^(e-56) is reproduced exactly:
    # 0.3 + 2^-20 lies in [2^-2, 2^-1), so e = 0 and its last bit is 2^-54
    x = 0.3 + 2.0 ** -20
    Q1, e1 = emu.split(np.array([[x]]))
    assert e1[0] == 0
    assert sum(Fraction(int(Q1[t, 0, 0])) * Fraction(2) ** (-7 * (t + 1)) for t in range(emu.NS)) == Fraction(x)


def test_balancing_keeps_row_products():
    rng = np.random.default_rng(4)
    A = rng.normal(size=(50, 3))
    B = rng.normal(size=(50, 3)) * 10.0 ** rng.uniform(-8, 8, (50, 1))
    a = emu.balance(A, B)
    np.testing.assert_array_equal(np.ldexp(A, a[:, None]) * np.ldexp(B, -a[:, None]), A * B)
    # the balanced row maxima differ by at most a factor 4 in exponent terms
    la = np.frexp(np.abs(np.ldexp(A, a[:, None])).max(1))[1]
    lb = np.frexp(np.abs(np.ldexp(B, -a[:, None])).max(1))[1]
    assert np.all(np.abs(la - lb) <= 1)
