"""Task graphs of the paper's workloads, built through the C ABI.

* tiled Cholesky (section "Numerical applications": POTRF on diagonal tiles,
  TRSM, SYRK and GEMM on the others), right-looking, k outer, followed by the
  block forward and back solves of A X = B;
* tiled GEMM C += A B with one task per (i, j, k) depending on the block C_ij
  (same section).

Matrices are row-major torch CUDA tensors; tiles are views (ld = row stride).
The graph refers to the tensors' memory; the caller keeps them alive until
the graph has been waited for.
"""
from __future__ import annotations

from . import spx


def _tiles_of(g: spx.Graph, M, b: int, lower_only: bool):
    n_r, n_c = M.shape
    Tr, Tc = -(-n_r // b), -(-n_c // b)
    h = {}
    for i in range(Tr):
        for j in range(Tc):
            if lower_only and j > i:
                continue
            v = M[i * b:(i + 1) * b, j * b:(j + 1) * b]
            h[i, j] = g.register_tensor(v)
    return h


def cholesky_graph(g: spx.Graph, A, b: int, X=None, lookahead: bool = True):
    """Insert the tasks of A = L L^T (lower, in place) and, when X is given,
    of the solve A Y = X (Y written over X).  Returns the number of tasks.

    Priorities (a scheduler hint, section "Task insertion"): with lookahead,
    POTRF, TRSM, SYRK and the GEMMs that update the next panel column go to
    the high-priority queue."""
    n = A.shape[0]
    T = -(-n // b)
    ta = _tiles_of(g, A, b, lower_only=True)
    R, W = spx.READ, spx.WRITE
    hi = 1 if lookahead else 0
    ntask = 0
    for k in range(T):
        t = g.insert(spx.OP_POTRF, [ta[k, k]], [W], priority=hi)
        g.set_arg(t, k * b)
        ntask += 1
        for i in range(k + 1, T):
            g.insert(spx.OP_TRSM, [ta[k, k], ta[i, k]], [R, W], priority=hi)
            ntask += 1
        for i in range(k + 1, T):
            g.insert(spx.OP_SYRK, [ta[i, k], ta[i, i]], [R, W], priority=hi)
            ntask += 1
        for j in range(k + 1, T):
            for i in range(j + 1, T):
                g.insert(spx.OP_GEMM_NT_SUB, [ta[i, k], ta[j, k], ta[i, j]], [R, R, W],
                         priority=hi if j == k + 1 else 0)
                ntask += 1
    if X is not None:
        tx = {}
        for i in range(T):
            tx[i] = g.register_tensor(X[i * b:(i + 1) * b, :])
        for k in range(T):
            g.insert(spx.OP_TRSM_L_FWD, [ta[k, k], tx[k]], [R, W], priority=hi)
            ntask += 1
            for i in range(k + 1, T):
                g.insert(spx.OP_GEMM_FWD, [ta[i, k], tx[k], tx[i]], [R, R, W])
                ntask += 1
        for k in range(T - 1, -1, -1):
            g.insert(spx.OP_TRSM_LT_BWD, [ta[k, k], tx[k]], [R, W], priority=hi)
            ntask += 1
            for i in range(k - 1, -1, -1):
                g.insert(spx.OP_GEMM_BWD, [ta[k, i], tx[k], tx[i]], [R, R, W])
                ntask += 1
    return ntask


def gemm_graph(g: spx.Graph, A, B, C, b: int, commutative: bool = False):
    """Insert the tasks of C += A B, one per (i, j, k), i and j outer, k inner."""
    n = A.shape[0]
    T = -(-n // b)
    ta = _tiles_of(g, A, b, False)
    tb = _tiles_of(g, B, b, False)
    tc = _tiles_of(g, C, b, False)
    mode = spx.COMMUTATIVE_WRITE if commutative else spx.WRITE
    for i in range(T):
        for j in range(T):
            for k in range(T):
                g.insert(spx.OP_GEMM_NN_ADD, [ta[i, k], tb[k, j], tc[i, j]], [spx.READ, spx.READ, mode])
    return T ** 3


def cholesky_flops(n: int, nrhs: int = 0) -> float:
    """Algorithmic flops: n^3/3 for the factorization (leading order, exact
    for the tiled task counts) plus 2 n^2 per right-hand side for the solve."""
    return n ** 3 / 3.0 + 2.0 * n * n * nrhs
