"""CPU ORACLE — FP64 products by splitting (the Ozaki scheme).  Test
infrastructure, not part of the product: only the test-suite, the smoke
check and the benchmark's CPU-baseline leg may import it.

The trailing updates of the paper's tiled Cholesky (section "Numerical
applications": SYRK and GEMM tasks) can run in FP64 emulated on BF16 tensor
cores by the error-free splitting of Ozaki, Ogita, Oishi and Rump ("Error-free
transformations of matrix multiplication by using fast routines of matrix
multiplication and its applications", Numer. Algorithms 59, 2012).  This
module states, in plain Python and numpy, the variant the library computes:

split(A), per row r of an FP64 matrix:
    e_r  = the smallest integer e >= -1022 with |a_rk| < 2^e for every k;
    X_rk = a_rk * 2^(55 - e_r) rounded to the nearest integer, ties to even;
    X_rk = sum_{s=0..7} sigma_s[r,k] * 128^(7-s), balanced digits taken from
           the least significant end: sigma = ((X + 64) mod 128) - 64, then
           X <- (X - sigma) / 128; what remains after seven digits is sigma_0.

gemm_nt_sub(C, A, B) = C - A B^T entry by entry (gemm_nn_add(C, A, B) = C +
A B the same way, with the columns of B split), v_rc the split product:
    P_d  = sum over s + t = d (d = 0..7) of sigma_s(A) tau_t(B)^T;
    F    = sum_d P_d * 128^(7-d)                    (an exact integer);
    v_rc = F * 2^(e_r + f_c - 61), rounded once to FP64;
    C_rc - v_rc rounded once.
(Since a ~ X 2^(e - 55) and b ~ Y 2^(f - 55), a b ~ X Y 2^(e + f - 110) and
X Y = 2^49 * sum_d P_d 128^(7-d) plus the dropped pairs s + t > 7.)

Pinned in tests/test_oracle_ozaki.py against a hand-worked split, exact
integer products, a closed-form worst case of the digit sums, and the exact
rational product within the error bound of the scheme; the NN form against
exact integer products and the exact scaling of single columns of B.
"""
from __future__ import annotations

import math

import numpy as np

PLANES = 8


def split(A):
    """(e, D): e int64 [rows] the row exponents, D int64 [8, rows, cols] the
    balanced base-128 digits of X = round(a 2^(55 - e))."""
    A = np.asarray(A, np.float64)
    rows, cols = A.shape
    e = np.empty(rows, np.int64)
    D = np.zeros((PLANES, rows, cols), np.int64)
    for r in range(rows):
        m = float(np.max(np.abs(A[r]))) if cols else 0.0
        # m = f 2^x with 1/2 <= f < 1: m < 2^x and m >= 2^(x-1)
        er = max(math.frexp(m)[1], -1022) if m > 0.0 else -1022
        e[r] = er
        # the scaling by a power of two is exact; a result below the normal
        # range is below 1/2 and rounds to zero either way
        X = np.rint(np.ldexp(A[r], 55 - er)).astype(np.int64)
        for s in range(PLANES - 1, 0, -1):
            d = (X + 64) % 128 - 64
            D[s, r] = d
            X = (X - d) // 128
        D[0, r] = X
    return e, D


def digit_sums(DA, DB):
    """P[d] = sum over s + t = d of DA[s] DB[t]^T, d = 0..7, as int64.  The
    FP64 matrix products are exact: every product and partial sum is an
    integer far below 2^53."""
    K = DA.shape[2]
    P = []
    for d in range(PLANES):
        acc = np.zeros((DA.shape[1], DB.shape[1]), np.float64)
        for s in range(d + 1):
            acc += DA[s].astype(np.float64) @ DB[d - s].astype(np.float64).T
        assert np.all(np.abs(acc) < 2.0 ** 53), K
        P.append(acc.astype(np.int64))
    return P


def products(A, B):
    """v[r, c]: the split product of row r of A and row c of B (FP64)."""
    eA, DA = split(A)
    eB, DB = split(B)
    P = digit_sums(DA, DB)
    F = np.zeros(P[0].shape, dtype=object)
    for d in range(PLANES):
        F = F + P[d].astype(object) * (128 ** (PLANES - 1 - d))
    v = np.empty(F.shape, np.float64)
    for (r, c), f in np.ndenumerate(F):
        # float(int) rounds to nearest even; the power-of-two scale is exact
        v[r, c] = math.ldexp(float(f), int(eA[r] + eB[c] - 61))
    return v


def gemm_nt_sub(C, A, B):
    """C - A B^T by the split product (a new array)."""
    return np.asarray(C, np.float64) - products(A, B)


def gemm_nn_add(C, A, B):
    """C + A B by the split product (a new array): A split by rows, B by
    columns (the rows of B^T, each column with its own exponent)."""
    return np.asarray(C, np.float64) + products(A, np.asarray(B, np.float64).T)


def tiled_gemm_nn_add(A, B, C, b):
    """The tiled GEMM C += A B of the paper's numerical applications with each
    task's product split: for every block C_ij, the tasks k = 0, 1, ... in
    order, each adding its split product with one rounding (in place)."""
    n = A.shape[0]
    T = -(-n // b)
    for i in range(T):
        for j in range(T):
            ri, cj = slice(i * b, min(n, (i + 1) * b)), slice(j * b, min(n, (j + 1) * b))
            for k in range(T):
                rk = slice(k * b, min(n, (k + 1) * b))
                C[ri, cj] = gemm_nn_add(C[ri, cj], A[ri, rk], B[rk, cj])
    return C


def syrk_lower(C, L):
    """C - L L^T on and below the diagonal, the strict upper part unchanged."""
    out = np.array(C, np.float64, copy=True)
    v = products(L, L)
    low = np.tril(np.ones(out.shape, bool))
    out[low] = out[low] - v[low]
    return out
