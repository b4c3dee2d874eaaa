"""Pins of the oracle's FP64 arithmetic against facts other than itself.

* diagonal matrices with power-of-4 entries and the identity: IEEE sqrt is
  exact, so L = diag(2^e) bit-exactly;
* A = L0 L0^T with L0 unit lower and entries in {-1, 0, 1}: every
  intermediate is an integer below 2^53, so any summation order returns L0
  bit-exactly, and the solve of A x = A x0 returns x0 bit-exactly;
* LAPACK (numpy.linalg.cholesky) and numpy's solve within FP64 bounds;
* tiled vs untiled oracle (different summation order) within 1e-13;
* backward errors <= 1e-14 on the small synthetic workload;
* non-SPD inputs report the LAPACK info column;
* the metrics are zero on exact factors and grow with planted errors;
* the tiled GEMM DAG equals the untiled triple loop bit for bit (same order of
  the k sum) and numpy's matmul within FP64 bounds.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2308_15964_b300 import inputs


def unit_lower(n, seed):
    rng = np.random.default_rng(seed)
    L = np.tril(rng.integers(-1, 2, size=(n, n)).astype(np.float64), -1)
    np.fill_diagonal(L, 1.0)
    return L


def lower(a):
    return np.tril(a)


@pytest.mark.parametrize("n,b", [(1, 1), (7, 7), (64, 16), (100, 32), (130, 64)])
def test_diagonal_power_of_four(n, b):
    e = (np.arange(n) % 9) - 4
    A = np.diag(4.0 ** e)
    L = A.copy()
    assert O.tiled_cholesky(L, b) == 0
    assert np.array_equal(lower(L), np.diag(2.0 ** e))
    L2 = A.copy()
    assert O.potrf(L2) == 0
    assert np.array_equal(lower(L2), np.diag(2.0 ** e))


@pytest.mark.parametrize("n,b,nrhs", [(48, 16, 1), (96, 32, 3), (100, 24, 2), (64, 64, 1)])
def test_integer_factor_exact(n, b, nrhs):
    L0 = unit_lower(n, n)
    A = L0 @ L0.T                        # exact: integer entries |a| <= n
    x0 = np.random.default_rng(1).integers(-3, 4, size=(n, nrhs)).astype(np.float64)
    B = A @ x0
    L = A.copy()
    X = B.copy()
    assert O.tiled_cholesky(L, b, X) == 0
    assert np.array_equal(lower(L), L0)
    assert np.array_equal(X, x0)
    # the strict upper triangle of the diagonal tiles is untouched
    T = -(-n // b)
    for k in range(T):
        r = slice(k * b, min(n, k * b + b))
        assert np.array_equal(np.triu(L[r, r], 1), np.triu(A[r, r], 1))
    L2 = A.copy()
    X2 = B.copy()
    assert O.potrf(L2) == 0
    O.solve_untiled(L2, X2)
    assert np.array_equal(lower(L2), L0) and np.array_equal(X2, x0)


def test_against_lapack_and_tiled_vs_untiled():
    n, b = 512, 64
    A = inputs.spd_matrix(n, 1.0, seed=1).numpy()
    Bv = inputs.rhs(n, 1, seed=1).numpy()
    Lt, X = A.copy(), Bv.copy()
    assert O.tiled_cholesky(Lt, b, X) == 0
    Lu = A.copy()
    assert O.potrf(Lu) == 0
    Llapack = np.linalg.cholesky(A)
    eps = np.abs(lower(Lt) - Llapack).max() / np.abs(Llapack).max()
    assert eps <= 1e-13
    eps_tu = np.abs(lower(Lt) - lower(Lu)).max() / np.abs(lower(Lu)).max()
    assert eps_tu <= 1e-13
    assert O.factor_backward_error(A, Lt) <= 1e-14
    eta = O.solve_backward_error(A, X, Bv)
    assert eta.max() <= 1e-14
    xs = np.linalg.solve(A, Bv)
    assert np.abs(X - xs).max() / np.abs(xs).max() <= 1e-12


@pytest.mark.parametrize("n,b", [(96, 32), (100, 32), (33, 8)])
def test_ragged_tiles(n, b):
    A = inputs.spd_matrix(n, 1.0, seed=11).numpy()
    Bv = inputs.rhs(n, 2, seed=11).numpy()
    L, X = A.copy(), Bv.copy()
    assert O.tiled_cholesky(L, b, X) == 0
    assert np.abs(lower(L) - np.linalg.cholesky(A)).max() <= 1e-13
    assert O.solve_backward_error(A, X, Bv).max() <= 1e-14


def test_not_spd_info():
    n, b = 96, 32
    A = np.eye(n)
    A[70, 70] = -1.0                    # pivot of global column 71 fails
    L = A.copy()
    assert O.tiled_cholesky(L, b) == 71
    L2 = A.copy()
    assert O.potrf(L2) == 71
    A = np.eye(n)
    A[5, 5] = np.nan
    assert O.tiled_cholesky(A.copy(), b) == 6
    A = inputs.spd_matrix(64, 1.0, seed=3).numpy()
    A[40, 40] = -5.0
    assert O.tiled_cholesky(A.copy(), 16) == O.potrf(A.copy()) == 41


def test_metrics_zero_and_planted():
    n = 64
    L0 = unit_lower(n, 5)
    A = L0 @ L0.T
    assert O.factor_backward_error(A, L0) == 0.0
    v = inputs.gaussian(n, 9)
    assert O.freivalds(A, L0, v) <= 1e-16     # only the rounding of L^T v
    x0 = np.ones((n, 1))
    assert O.solve_backward_error(A, x0, A @ x0).max() == 0.0
    Lbad = L0.copy()
    Lbad[40, 3] += 1e-6
    assert O.factor_backward_error(A, Lbad) > 1e-9
    assert O.freivalds(A, Lbad, v) > 1e-10
    xbad = x0.copy()
    xbad[7, 0] += 1e-6
    assert O.solve_backward_error(A, xbad, A @ x0).max() > 1e-9
    # closed form: a single perturbed entry d of L gives ||A - LL^T||_F of
    # roughly sqrt(2) * d * ||row|| -- check the order of magnitude only
    d = 1e-6
    beta = O.factor_backward_error(A, Lbad)
    assert 0.1 * d / np.linalg.norm(A) < beta < 100 * d * n / np.linalg.norm(A)


def test_solve_backward_error_closed_form():
    """Rigal-Gaches eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)
    on a hand-worked 3 x 3 case.  A is not symmetric, so its infinity norm
    (max row sum 5) differs from its 1-norm (max column sum 6); each x has
    ||x||_1 != ||x||_inf; b = A x + d with d exactly representable, so the
    residual is exactly d.  By hand:
      column 0: x = (1, -2, 3), A x = (6, -2, 7), d = (0, 1/2, 0),
                b = (6, -3/2, 7): eta = (1/2) / (5*3 + 7) = 1/44;
      column 1: x = (-3, 0, 1), A x = (-12, -2, 1), d = (-1/4, 0, 1/8),
                b = (-49/4, -2, 9/8): eta = (1/4) / (5*3 + 49/4) = 1/109.
    A 1-norm of A would give 1/50 and 1/121; ||x||_1 1/74 and 1/129; a dropped
    ||b|| term 1/30 and 1/60; the residual of a wrong sign or a transposed A
    changes the numerators."""
    A = np.array([[4.0, -1.0, 0.0], [1.0, 3.0, 1.0], [0.0, -2.0, 1.0]])
    X = np.array([[1.0, -3.0], [-2.0, 0.0], [3.0, 1.0]])
    B = np.array([[6.0, -12.25], [-1.5, -2.0], [7.0, 1.125]])
    eta = O.solve_backward_error(A, X, B)
    assert eta[0] == 1.0 / 44.0 and eta[1] == 1.0 / 109.0, eta


@pytest.mark.parametrize("n,b", [(64, 16), (96, 32), (70, 32)])
def test_gemm_dag_exact_order(n, b):
    A = inputs.uniform((n, n), 3).numpy()
    B = inputs.uniform((n, n), 4).numpy()
    C = inputs.uniform((n, n), 5).numpy()
    Ct, Cu = C.copy(), C.copy()
    assert O.tiled_gemm(A, B, Ct, b) == 0
    O.gemm_untiled(A, B, Cu)
    assert np.array_equal(Ct, Cu)
    ref = C + A @ B
    assert np.abs(Ct - ref).max() <= 4 * n * 2.2e-16 * (np.abs(A) @ np.abs(B)).max()
    Cc = C.copy()
    assert O.tiled_gemm(A, B, Cc, b, commutative=True) == 0
    assert np.array_equal(Cc, Cu)


def test_generator_bits():
    # splitmix64 against its scalar definition; exactness of the SPD recipe
    import torch
    c = torch.arange(0, 50, dtype=torch.int64)
    got = inputs.splitmix64(c, 12345).numpy().view(np.uint64)
    ref = np.array([inputs.splitmix64_ref(12345, i) for i in range(50)], dtype=np.uint64)
    assert np.array_equal(got, ref)
    # first outputs of splitmix64 seeded with 0 (published test vector of the
    # reference implementation, Vigna's splitmix64.c with x = 0)
    assert inputs.splitmix64_ref(0, 0) == 0xE220A8397B1DCDAF
    assert inputs.splitmix64_ref(0, 1) == 0x6E789E6AA1B965F4
    u = inputs.uniform((10000,), 7).numpy()
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.05
    n = 96
    A = inputs.spd_matrix(n, 0.5, 2).numpy()
    assert np.array_equal(A, A.T)
    K = inputs.int_lattice(n, n, 2).numpy()
    assert K.min() >= -127 and K.max() <= 127
    G = K @ K.T
    ref = G / float(127 * 127 * n)
    ref[np.diag_indices(n)] += 0.5
    assert np.array_equal(A, ref)


# ---------------------------------------------------------------------------
# Inverses of the diagonal tiles and the block solve that applies them.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 5, 40])
def test_trtri_integer_unit_lower_exact(n):
    # the inverse of an integer unit-lower matrix is an integer unit-lower
    # matrix; every intermediate is an exact integer
    L = unit_lower(n, 3 * n)
    V = O.trtri(L)
    assert np.array_equal(L @ V, np.eye(n))
    assert np.array_equal(V, np.round(V))
    assert np.array_equal(np.triu(V, 1), np.zeros((n, n)))


def test_trtri_power_of_two_diagonal():
    e = (np.arange(30) % 11) - 5
    V = O.trtri(np.diag(2.0 ** e))
    assert np.array_equal(V, np.diag(2.0 ** -e))


def test_trtri_against_numpy():
    A = inputs.spd_matrix(96, 1.0, seed=11).numpy()
    L = np.linalg.cholesky(A)
    V = O.trtri(L)
    Vn = np.linalg.inv(L)
    assert np.abs(V - Vn).max() <= 1e-13 * np.abs(Vn).max()
    assert np.abs(L @ V - np.eye(96)).max() <= 1e-14


def _solve_inv(L, R, b):
    """Oracle block solve with the diagonal inverses: R in, R out."""
    n, nrhs = R.shape
    T = -(-n // b)
    V = np.zeros((n, b))
    D = np.zeros_like(R)
    Lc = np.ascontiguousarray(L)
    assert O.execute(O.trtri_tasks(T), {"A": Lc, "V": V}, b) == 0
    assert O.execute(O.solve_inv_tasks(T), {"A": Lc, "V": V, "R": R, "D": D}, b) == 0
    return V


@pytest.mark.parametrize("n,b,nrhs", [(48, 16, 1), (100, 32, 3), (64, 64, 2)])
def test_solve_inv_integer_exact(n, b, nrhs):
    L0 = unit_lower(n, n + 7)
    A = L0 @ L0.T
    x0 = np.random.default_rng(2).integers(-3, 4, size=(n, nrhs)).astype(np.float64)
    L = A.copy()
    assert O.tiled_cholesky(L, b) == 0
    R = A @ x0
    V = _solve_inv(lower(L), R, b)
    assert np.array_equal(R, x0)
    # V holds the inverse of each diagonal tile (ragged last tile included)
    for k in range(-(-n // b)):
        r = slice(k * b, min(n, k * b + b))
        m = r.stop - r.start
        assert np.array_equal(V[r, :m] @ L0[r, r], np.eye(m))


@pytest.mark.parametrize("n,b", [(200, 64), (130, 32)])
def test_solve_inv_matches_substitution(n, b):
    A = inputs.spd_matrix(n, 1.0, seed=n).numpy()
    B = inputs.rhs(n, 3, seed=n).numpy()
    L = A.copy()
    assert O.tiled_cholesky(L, b) == 0
    L = lower(L)
    X1 = B.copy()
    O.solve_untiled(np.ascontiguousarray(L), X1)
    X2 = B.copy()
    _solve_inv(L, X2, b)
    assert np.abs(X1 - X2).max() <= 1e-12 * np.abs(X1).max()
    assert O.solve_backward_error(A, X2, B).max() <= 1e-14


def test_trmm_plain_product():
    rng = np.random.default_rng(5)
    n, r = 24, 4
    T = np.tril(rng.uniform(-1, 1, (n, n)))
    X = rng.uniform(-1, 1, (n, r))
    for arg, ref in ((0, T @ X), (1, T.T @ X)):
        V = np.ascontiguousarray(T)
        R = X.copy()
        D = np.zeros_like(X)
        tasks = [(O.TRMM, [(("V", 0), O.READ), (("R", 0), O.READ), (("D", 0), O.WRITE)], arg)]
        assert O.execute(tasks, {"V": V, "R": R, "D": D}, n) == 0
        assert np.abs(D - ref).max() <= 1e-14 * n


@pytest.mark.parametrize("n,b", [(64, 16), (80, 32), (48, 48)])
def test_cholesky_inv_integer_exact(n, b):
    """The Cholesky whose panel solves apply the inverse of the diagonal tile
    (TRTRI, then A_ik <- A_ik V_k^T): for A = L0 L0^T with L0 unit lower and
    entries in {-1, 0, 1}, every intermediate (the inverses included, whose
    entries stay far below 2^53 at these tile sizes) is an integer, so the
    factor is L0 exactly and V holds the exact inverses of its diagonal
    tiles.  A transposed or misplaced V fails this."""
    L0 = unit_lower(n, n + b)
    A = L0 @ L0.T
    V = np.zeros((n, b), np.float64)
    assert O.tiled_cholesky_inv(A, b, V) == 0
    assert np.array_equal(np.tril(A), L0)
    for k in range(0, n, b):
        bk = min(b, n - k)
        blk = L0[k:k + bk, k:k + bk]
        assert np.array_equal(V[k:k + bk, :bk] @ blk, np.eye(bk))


@pytest.mark.parametrize("n,b", [(96, 32), (100, 32), (128, 64)])
def test_cholesky_inv_matches_substitution(n, b):
    """On a random SPD matrix the inverse-based panel solve gives the factor
    of the substitution form (itself pinned above) to FP64 rounding, and
    TRSM_INV(TRTRI(L_kk), A_ik) equals TRSM(L_kk, A_ik) tile by tile."""
    A = inputs.spd_matrix(n, 0.1, seed=n).numpy()
    L1, L2 = A.copy(), A.copy()
    V = np.zeros((n, b), np.float64)
    assert O.tiled_cholesky(L1, b) == 0
    assert O.tiled_cholesky_inv(L2, b, V) == 0
    err = np.abs(np.tril(L1) - np.tril(L2)).max() / np.abs(np.tril(L1)).max()
    assert err <= 1e-13, err


def test_axpy_f32_exact():
    """FP32 y <- y + alpha x, one rounding per operation: numpy's float32
    arithmetic (IEEE single, no fused multiply-add) gives the same bits;
    alpha = 1 adds x directly; small integers and powers of two are exact."""
    n = 100003
    x = inputs.uniform((n,), 11).numpy().astype(np.float32)
    y0 = inputs.uniform((n,), 12).numpy().astype(np.float32)
    for alpha in (1.0, 0.5, -3.25, 1.1):
        y = y0.copy()
        O.axpy_f32(x, y, alpha)
        a = np.float32(alpha)
        ref = (y0 + x) if alpha == 1.0 else (a * x + y0)
        assert ref.dtype == np.float32
        assert np.array_equal(y, ref), alpha
    xi = np.arange(-50, 50, dtype=np.float32)
    yi = np.full(100, 7.0, np.float32)
    O.axpy_f32(xi, yi, 2.0)
    assert np.array_equal(yi, 2 * np.arange(-50, 50) + 7.0)


def particles(sizes, seed):
    N = int(np.sum(sizes))
    P = np.zeros((N, 8), np.float64)
    P[:, 0:3] = inputs.uniform((N, 3), seed).numpy()
    P[:, 3] = inputs.uniform((N,), seed + 1).numpy()
    return np.ascontiguousarray(P)


def test_nbody_closed_forms():
    """Two charges 2 and 3 at distance 2 on the x axis: phi = 3/2 and 1, E_x =
    3 (0 - 2) / 8 = -3/4 and 2 (2 - 0) / 8 = 1/2, exactly.  Six unit charges
    at +-e_x, +-e_y, +-e_z around a charge at the origin: phi = 6 and E = 0
    exactly at the origin (the terms cancel pairwise in order)."""
    P = np.zeros((2, 8))
    P[0, 3], P[1, 0], P[1, 3] = 2.0, 2.0, 3.0
    assert O.nbody(P, [2]) == 0
    assert P[0, 4] == 1.5 and P[1, 4] == 1.0
    assert P[0, 5] == -0.75 and P[1, 5] == 0.5 and not P[:, 6:].any()
    Q = np.zeros((7, 8))
    Q[0, 3] = 1.0
    for k, (ax, sg) in enumerate([(0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1)]):
        Q[k + 1, ax] = sg
        Q[k + 1, 3] = 1.0
    Q2 = Q.copy()
    assert O.nbody(Q, [7]) == 0
    assert Q[0, 4] == 6.0 and not Q[0, 5:].any()
    # the same particles in two groups (pair tasks): same values
    assert O.nbody(Q2, [3, 4]) == 0
    assert Q2[0, 4] == 6.0 and not Q2[0, 5:].any()


@pytest.mark.parametrize("sizes", [[40], [7, 30, 13], [1, 1, 5]])
def test_nbody_vs_numpy_and_newton(sizes):
    """Random charges: the grouped task list equals the all-pairs sum (numpy
    broadcasting over the definition) to FP64 rounding, and the total force
    sum_i q_i E_i vanishes (Newton's third law) to rounding."""
    P = particles(sizes, sum(sizes))
    X, q = P[:, :3].copy(), P[:, 3].copy()
    assert O.nbody(P, sizes) == 0
    d = X[:, None, :] - X[None, :, :]
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    phi = (q[None, :] / r).sum(1)
    E = (q[None, :, None] * d / r[:, :, None] ** 3).sum(1)
    scale = (np.abs(q)[None, :] / r ** 2).sum(1).max() * len(q)
    assert np.abs(P[:, 4] - phi).max() <= 1e-13 * np.abs(phi).max()
    assert np.abs(P[:, 5:] - E).max() <= 1e-13 * scale
    total = (q[:, None] * P[:, 5:]).sum(0)
    assert np.abs(total).max() <= 1e-12 * scale
