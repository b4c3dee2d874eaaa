"""Pins of the oracle's split (Ozaki) FP64 product against facts other than
itself:

* a hand-worked split (exponents and digits worked out on paper), including
  the extreme top digit 64 and a negative bottom digit from the balancing;
* the digits rebuild X = round(a 2^(55 - e)) exactly (Python integers) and X
  2^(e - 55) is within 2^(e - 56) of a, equal to a when ulp(a) >= 2^(e - 55);
* products of integer matrices below 2^19 are exact (their digits stop at
  plane 3, so no pair is dropped), equal to the integer product;
* the worst case of the digit sums (every digit -64, the top one -63, K = 512)
  against a closed form for every P_d, P_7 just below 2^24;
* the exact rational product (fractions.Fraction) within the error bound of
  the scheme: K * 9.1 * 2^-56 * 2^(e_r + f_c) plus the final rounding.  A
  dropped pair s + t = 7 breaks it on the worst case above.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import ozaki as Z


def test_split_hand_worked():
    # row max 1.0 -> e = 1: X(1.0) = 2^54 = 32 * 128^7; X(-0.75) = -24 * 128^7;
    # X(2^-60) = 2^-6 rounds to 0
    e, D = Z.split(np.array([[1.0, -0.75, 2.0 ** -60, 0.0]]))
    assert e[0] == 1
    assert D[:, 0, 0].tolist() == [32, 0, 0, 0, 0, 0, 0, 0]
    assert D[:, 0, 1].tolist() == [-24, 0, 0, 0, 0, 0, 0, 0]
    assert D[:, 0, 2].tolist() == [0] * 8
    # 0.5 + 2^-8: e = 0, X = 2^54 + 2^47 = 32 * 128^7 + 32 * 128^6
    e, D = Z.split(np.array([[0.5 + 2.0 ** -8]]))
    assert e[0] == 0 and D[:, 0, 0].tolist() == [32, 32, 0, 0, 0, 0, 0, 0]
    # 0.5 - 2^-54 < 1/2: e = -1, X = 2^55 - 4 = 64 * 128^7 - 4: the balanced
    # bottom digit is -4 and the top digit reaches 64
    e, D = Z.split(np.array([[0.5 - 2.0 ** -54]]))
    assert e[0] == -1 and D[:, 0, 0].tolist() == [64, 0, 0, 0, 0, 0, 0, -4]
    # zero row and a subnormal row take e = -1022
    e, D = Z.split(np.array([[0.0, 0.0], [5e-324, -1e-310]]))
    assert e.tolist() == [-1022, -1022] and not D[:, 0].any()
    X = sum(int(D[s, 1, 1]) * 128 ** (7 - s) for s in range(8))
    assert Fraction(X) * Fraction(2) ** (-1022 - 55) == Fraction(-1e-310)


@pytest.mark.parametrize("seed", range(4))
def test_split_rebuilds(seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((12, 40)) * np.exp2(rng.integers(-60, 60, size=(12, 1)))
    A[3, :] = 0.0
    A[5, 7] = 0.0
    A[6] *= np.exp2(rng.integers(-40, 0, size=40))  # a row of spread magnitudes
    e, D = Z.split(A)
    assert D[1:].min() >= -64 and D[1:].max() <= 63
    assert D[0].min() >= -64 and D[0].max() <= 64
    for r in range(A.shape[0]):
        m = np.abs(A[r]).max()
        assert m < 2.0 ** e[r]
        assert e[r] == -1022 or m >= 2.0 ** (e[r] - 1)
        for k in range(A.shape[1]):
            X = sum(int(D[s, r, k]) * 128 ** (7 - s) for s in range(8))
            a = Fraction(float(A[r, k]))
            scaled = a * Fraction(2) ** (55 - int(e[r]))
            assert abs(Fraction(X) - scaled) <= Fraction(1, 2)
            back = Fraction(X) * Fraction(2) ** (int(e[r]) - 55)
            assert abs(back - a) <= Fraction(2) ** (int(e[r]) - 56)
            if scaled.denominator == 1:
                assert back == a


@pytest.mark.parametrize("K", [1, 16, 64, 512])
def test_integer_products_exact(K):
    rng = np.random.default_rng(K)
    A = rng.integers(-2 ** 19, 2 ** 19, size=(17, K))
    B = rng.integers(-2 ** 19, 2 ** 19, size=(9, K))
    exact = A @ B.T  # int64: |sum| < 512 * 2^38
    v = Z.products(A.astype(np.float64), B.astype(np.float64))
    assert np.array_equal(v, exact.astype(np.float64))
    C = rng.integers(-2 ** 40, 2 ** 40, size=(17, 9))
    assert np.array_equal(Z.gemm_nt_sub(C.astype(np.float64), A.astype(np.float64),
                                        B.astype(np.float64)), (C - exact).astype(np.float64))


def worst_case_row(K):
    """A row whose digits are all -64 except sigma_0 = -63 (e = 0)."""
    X = 63 * 128 ** 7 + 64 * sum(128 ** j for j in range(7))
    a = -float(Fraction(X, 2 ** 55))
    assert Fraction(a) == -Fraction(X, 2 ** 55)  # 49 significant bits
    return np.full((1, K), a)


def test_worst_case_digit_sums():
    K = 512
    A = worst_case_row(K)
    e, D = Z.split(A)
    assert e[0] == 0 and D[:, 0, 0].tolist() == [-63] + [-64] * 7
    P = Z.digit_sums(D, D)
    # d = 0: 63^2 per k; d >= 1: the two pairs with an index 0 give 63 * 64,
    # the d - 1 others 64^2
    want = [K * 63 * 63] + [K * (2 * 63 * 64 + (d - 1) * 64 * 64) for d in range(1, 8)]
    assert [int(p[0, 0]) for p in P] == want
    assert 2 ** 24 - 2 ** 17 < want[7] <= 2 ** 24
    F = sum(w * 128 ** (7 - d) for d, w in enumerate(want))
    assert Z.products(A, A)[0, 0] == float(Fraction(F, 2 ** 61))


def bound_check(A, B):
    v = Z.products(A, B)
    eA, _ = Z.split(A)
    eB, _ = Z.split(B)
    K = A.shape[1]
    worst = 0.0
    for r in range(A.shape[0]):
        for c in range(B.shape[0]):
            exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(A[r], B[c]))
            err = abs(Fraction(float(v[r, c])) - exact)
            bound = (Fraction(K * 91, 10) * Fraction(2) ** (int(eA[r] + eB[c]) - 56)
                     + abs(Fraction(float(v[r, c]))) * Fraction(2) ** -53)
            assert err <= bound, (r, c, float(err), float(bound))
            worst = max(worst, float(err / bound))
    return worst


@pytest.mark.parametrize("K", [8, 64, 512])
def test_error_bound_random(K):
    rng = np.random.default_rng(100 + K)
    A = rng.standard_normal((4, K)) * np.exp2(rng.integers(-30, 30, size=(4, 1)))
    B = rng.standard_normal((3, K)) * np.exp2(rng.integers(-30, 30, size=(3, 1)))
    bound_check(A, B)


def test_error_bound_worst_case_catches_dropped_pair():
    A = worst_case_row(512)
    bound_check(A, A)
    # the d = 7 term alone is far above the bound: dropping it would fail
    K = 512
    assert Fraction(K * (2 * 63 * 64 + 6 * 64 * 64), 2 ** 61) > Fraction(K * 91, 10) * Fraction(2) ** -56


def test_gemm_nn_add_integer_exact():
    """Integer A, B below 2^19: the NN split product is exact, so C + A B
    equals the integer sum (tiled too, whatever the tile size)."""
    rng = np.random.default_rng(11)
    A = rng.integers(-2 ** 19, 2 ** 19, size=(37, 70))
    B = rng.integers(-2 ** 19, 2 ** 19, size=(70, 45))
    C = rng.integers(-2 ** 40, 2 ** 40, size=(37, 45))
    want = (C + A @ B).astype(np.float64)
    got = Z.gemm_nn_add(C.astype(np.float64), A.astype(np.float64), B.astype(np.float64))
    assert np.array_equal(got, want)
    n = 70
    A2 = rng.integers(-2 ** 19, 2 ** 19, size=(n, n))
    B2 = rng.integers(-2 ** 19, 2 ** 19, size=(n, n))
    C2 = rng.integers(-2 ** 30, 2 ** 30, size=(n, n))
    for b in (32, 64):
        got = Z.tiled_gemm_nn_add(A2.astype(np.float64), B2.astype(np.float64),
                                  C2.astype(np.float64), b)
        assert np.array_equal(got, (C2 + A2 @ B2).astype(np.float64))


def test_gemm_nn_add_splits_columns_of_b():
    """Each column of B carries its own exponent: scaling column c of B by
    2^s scales column c of the product by exactly 2^s and leaves the others
    bit for bit.  A split of B by rows (a transposed operand) would mix the
    columns' magnitudes in one row exponent and fail both."""
    rng = np.random.default_rng(12)
    A = rng.standard_normal((9, 40))
    B = rng.standard_normal((40, 6))
    C = np.zeros((9, 6))
    base = Z.gemm_nn_add(C, A, B)
    for c, sh in ((0, 40), (3, -35), (5, 7)):
        B2 = B.copy()
        B2[:, c] *= 2.0 ** sh
        got = Z.gemm_nn_add(C, A, B2)
        assert np.array_equal(got[:, c], base[:, c] * 2.0 ** sh)
        others = [j for j in range(6) if j != c]
        assert np.array_equal(got[:, others], base[:, others])
    # and the result is within the scheme's bound of the exact product
    bound_check(A, np.ascontiguousarray(B.T))


def test_syrk_lower_matches_gemm():
    rng = np.random.default_rng(7)
    L = rng.standard_normal((20, 33))
    C = rng.standard_normal((20, 20))
    S = Z.syrk_lower(C, L)
    G = Z.gemm_nt_sub(C, L, L)
    low = np.tril(np.ones((20, 20), bool))
    assert np.array_equal(S[low], G[low])
    assert np.array_equal(S[~low], C[~low])
