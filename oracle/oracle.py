"""CPU ORACLE (Python side) — test infrastructure, not part of the product.

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this module.  It loads ``liboracle.so`` built from
``oracle/spx_oracle.cpp`` and adds the oracle's own task-list generators for
the paper's workloads (tiled Cholesky with POTRF/TRSM/SYRK/GEMM tasks, the
block solve, and the tiled GEMM whose tasks depend on the blocks of C; section
"Numerical applications").  It shares no code with the CUDA path; only the
seeded input generators (``paper_2308_15964_b300.inputs``) serve both.

Every function names the passage it follows.  Functions without a pin other
than themselves are marked "parity unpinned" (none at present).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
SRC = os.path.join(HERE, "spx_oracle.cpp")

READ, WRITE, COMMUTATIVE_WRITE, ATOMIC_WRITE, MAYBE_WRITE = 0, 1, 2, 3, 4
(POTRF, TRSM, SYRK, GEMM_NT_SUB, GEMM_NN_ADD, TRSM_L_FWD, GEMM_FWD,
 TRSM_LT_BWD, GEMM_BWD, NOP, SPIN, COPY, AXPY, TRMM, TRTRI, TRSM_INV, NBODY_SELF,
 NBODY_PAIR, POTRF_PANEL) = range(19)


def build(force: bool = False) -> str:
    """Compile the oracle with plain IEEE FP64 (no FMA contraction, no fast-math)."""
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC):
        return LIB_PATH
    os.makedirs(BUILD_DIR, exist_ok=True)
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.c_void_p
        L.spxo_derive.restype = ctypes.c_longlong
        L.spxo_derive.argtypes = [ctypes.c_int, ctypes.c_longlong, P, P, P, P, P, P, ctypes.c_longlong]
        L.spxo_potrf.restype = ctypes.c_int
        L.spxo_potrf.argtypes = [P, ctypes.c_int, ctypes.c_int]
        L.spxo_trsv_lower.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.spxo_trsv_lower_t.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.spxo_trtri.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int]
        L.spxo_execute.restype = ctypes.c_int
        L.spxo_execute.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_int, P]
        L.spxo_gemm_untiled.argtypes = [P, P, P, ctypes.c_int]
        L.spxo_factor_backward_error.restype = ctypes.c_double
        L.spxo_factor_backward_error.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int]
        L.spxo_solve_backward_error.argtypes = [P, ctypes.c_int, P, P, ctypes.c_int, ctypes.c_int, P]
        L.spxo_axpy_f32.argtypes = [ctypes.c_longlong, ctypes.c_float, P, P]
        L.spxo_freivalds.restype = ctypes.c_double
        L.spxo_freivalds.argtypes = [P, ctypes.c_int, P, ctypes.c_int, ctypes.c_int, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------------------
# DAG derivation (section "Internal implementation": per-address data handles
# with ordered dependency lists; section "Task insertion": access modes).
# ---------------------------------------------------------------------------

def derive(ntasks: int, task, key, mode):
    """Successor CSR (row_ptr, col, indeg) of an access list given in insertion order."""
    task = np.ascontiguousarray(task, dtype=np.uint32)
    key = np.ascontiguousarray(key, dtype=np.uint64)
    mode = np.ascontiguousarray(mode, dtype=np.int32)
    row_ptr = np.zeros(ntasks + 1, dtype=np.uint32)
    indeg = np.zeros(max(ntasks, 1), dtype=np.uint32)
    cap = max(16, 4 * len(task))
    while True:
        col = np.zeros(cap, dtype=np.uint32)
        ne = lib().spxo_derive(ntasks, len(task), _p(task), _p(key), _p(mode), _p(row_ptr),
                               _p(indeg), _p(col), cap)
        if ne < 0:
            raise ValueError("malformed access list")
        if ne <= cap:
            return row_ptr, col[:ne].copy(), indeg[:ntasks].copy()
        cap = int(ne)


# ---------------------------------------------------------------------------
# Task lists of the paper's workloads, written independently of the product.
# A task is (op, [(tile_name, mode), ...], arg).  Tile names are tuples.
# ---------------------------------------------------------------------------

def cholesky_tasks(T: int, b: int, with_solve: bool = False):
    """Right-looking tiled Cholesky, k outer (POTRF, TRSM, SYRK, GEMM; section
    "Numerical applications"), then the block forward solve (k ascending) and
    back solve (k descending) on one RHS panel.  arg of POTRF(k) = k*b, the
    global column offset used for the LAPACK-style info."""
    tasks = []
    for k in range(T):
        tasks.append((POTRF, [(("A", k, k), WRITE)], k * b))
        for i in range(k + 1, T):
            tasks.append((TRSM, [(("A", k, k), READ), (("A", i, k), WRITE)], 0))
        for i in range(k + 1, T):
            tasks.append((SYRK, [(("A", i, k), READ), (("A", i, i), WRITE)], 0))
        for j in range(k + 1, T):
            for i in range(j + 1, T):
                tasks.append((GEMM_NT_SUB, [(("A", i, k), READ), (("A", j, k), READ),
                                            (("A", i, j), WRITE)], 0))
    if with_solve:
        for k in range(T):
            tasks.append((TRSM_L_FWD, [(("A", k, k), READ), (("X", k), WRITE)], 0))
            for i in range(k + 1, T):
                tasks.append((GEMM_FWD, [(("A", i, k), READ), (("X", k), READ),
                                         (("X", i), WRITE)], 0))
        for k in range(T - 1, -1, -1):
            tasks.append((TRSM_LT_BWD, [(("A", k, k), READ), (("X", k), WRITE)], 0))
            for i in range(k - 1, -1, -1):
                tasks.append((GEMM_BWD, [(("A", k, i), READ), (("X", k), READ),
                                         (("X", i), WRITE)], 0))
    return tasks


def cholesky_inv_tasks(T: int, b: int):
    """The tiled Cholesky with the panel solves by the inverse of the diagonal
    tile: for k, POTRF(k), TRSM(k+1, k) by substitution, TRTRI(L_kk -> V_k),
    TRSM_INV(V_k, A_ik) for i > k + 1 (A_ik <- A_ik V_k^T, the same L_ik as
    TRSM up to rounding), then SYRK and GEMM as in cholesky_tasks."""
    tasks = []
    for k in range(T):
        tasks.append((POTRF, [(("A", k, k), WRITE)], k * b))
        if k + 1 < T:
            tasks.append((TRSM, [(("A", k, k), READ), (("A", k + 1, k), WRITE)], 0))
        tasks.append((TRTRI, [(("A", k, k), READ), (("V", k), WRITE)], 0))
        for i in range(k + 2, T):
            tasks.append((TRSM_INV, [(("V", k), READ), (("A", i, k), WRITE)], 0))
        for i in range(k + 1, T):
            tasks.append((SYRK, [(("A", i, k), READ), (("A", i, i), WRITE)], 0))
        for j in range(k + 1, T):
            for i in range(j + 1, T):
                tasks.append((GEMM_NT_SUB, [(("A", i, k), READ), (("A", j, k), READ),
                                            (("A", i, j), WRITE)], 0))
    return tasks


def tiled_cholesky_inv(A: np.ndarray, b: int, V: np.ndarray) -> int:
    """cholesky_inv_tasks on A in place; V (n x b) receives the inverses of
    the diagonal factor tiles.  Returns info."""
    n = A.shape[0]
    T = -(-n // b)
    return execute(cholesky_inv_tasks(T, b), {"A": A, "V": V}, b)


def trtri_tasks(T: int):
    """Inverse of every diagonal factor tile: V_k <- L_kk^{-1}."""
    return [(TRTRI, [(("A", k, k), READ), (("V", k), WRITE)], 0) for k in range(T)]


def solve_inv_tasks(T: int):
    """Block solve L L^T x = r with the inverses of the diagonal tiles applied
    as products (y_k = L_kk^{-1} (r_k - sum_j L_kj y_j), then x_k = L_kk^{-T}
    (y_k - sum_i L_ik^T x_i)).  The right-hand side starts in R; the forward
    sweep writes y into D, the backward sweep writes x back into R."""
    tasks = []
    for k in range(T):
        tasks.append((TRMM, [(("V", k), READ), (("R", k), READ), (("D", k), WRITE)], 0))
        for i in range(k + 1, T):
            tasks.append((GEMM_FWD, [(("A", i, k), READ), (("D", k), READ), (("R", i), WRITE)], 0))
    for k in range(T - 1, -1, -1):
        tasks.append((TRMM, [(("V", k), READ), (("D", k), READ), (("R", k), WRITE)], 1))
        for i in range(k - 1, -1, -1):
            tasks.append((GEMM_BWD, [(("A", k, i), READ), (("R", k), READ), (("D", i), WRITE)], 0))
    return tasks


def trtri(L: np.ndarray) -> np.ndarray:
    """Inverse of the lower triangle of L (untiled, forward substitution on
    the identity)."""
    n = L.shape[0]
    L = np.ascontiguousarray(L, np.float64)
    V = np.zeros((n, n), np.float64)
    lib().spxo_trtri(_p(L), L.shape[1], _p(V), n, n)
    return V


def gemm_tasks(T: int, commutative: bool = False, mode: int | None = None):
    """Tiled C += A B with one task per (i, j, k), i and j outer, k inner; each
    task depends on the block C_ij it updates (section "Numerical applications"),
    with a WRITE, a COMMUTATIVE_WRITE (commutative) or any given mode."""
    if mode is None:
        mode = COMMUTATIVE_WRITE if commutative else WRITE
    tasks = []
    for i in range(T):
        for j in range(T):
            for k in range(T):
                tasks.append((GEMM_NN_ADD, [(("A", i, k), READ), (("B", k, j), READ),
                                            (("C", i, j), mode)], 0))
    return tasks


def nbody_tasks(G: int, commutative: bool = False):
    """The particle test case: for each group i, the interactions inside it,
    then with every later group j (both groups written; section "Numerical
    applications": dependencies on whole groups)."""
    mode = COMMUTATIVE_WRITE if commutative else WRITE
    tasks = []
    for i in range(G):
        tasks.append((NBODY_SELF, [(("P", i), mode)], 0))
        for j in range(i + 1, G):
            tasks.append((NBODY_PAIR, [(("P", i), mode), (("P", j), mode)], 0))
    return tasks


def nbody(P: np.ndarray, sizes, commutative: bool = False) -> int:
    """Run nbody_tasks on the particles P (N x 8 FP64, groups of the given
    sizes stacked in order) in insertion order, accumulating phi and E."""
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    assert P.shape == (offs[-1], 8) and P.dtype == np.float64 and P.flags["C_CONTIGUOUS"]
    return execute(nbody_tasks(len(sizes), commutative), {"P": P}, 0, groups=offs)


def axpy_f32(x: np.ndarray, y: np.ndarray, alpha: float) -> None:
    """y <- y + alpha x in FP32 (the AXPY test case), in place."""
    assert x.dtype == np.float32 and y.dtype == np.float32 and x.shape == y.shape
    x = np.ascontiguousarray(x)
    assert y.flags["C_CONTIGUOUS"]
    lib().spxo_axpy_f32(ctypes.c_longlong(x.size), ctypes.c_float(alpha), _p(x), _p(y))


def access_arrays(tasks):
    """Flatten a task list to (task, key, mode) arrays; keys number tile names
    in order of first use."""
    names = {}
    t_arr, k_arr, m_arr = [], [], []
    for t, (_, acc, _) in enumerate(tasks):
        for name, mode in acc:
            if name not in names:
                names[name] = len(names)
            t_arr.append(t)
            k_arr.append(names[name])
            m_arr.append(mode)
    return (np.asarray(t_arr, np.uint32), np.asarray(k_arr, np.uint64),
            np.asarray(m_arr, np.int32), names)


# ---------------------------------------------------------------------------
# Tiled execution in insertion order (STF sequential semantics).
# ---------------------------------------------------------------------------

class _Tile(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("rows", ctypes.c_int), ("cols", ctypes.c_int),
                ("ld", ctypes.c_int), ("pad", ctypes.c_int)]


def _tile_views(names, mats, b, groups=None):
    """Tile table for named tiles ("A", i, j) / ("B", ...) / ("C", ...) of square
    row-major matrices, ("X", i) / ("R", i) / ("D", i) row blocks of n x nrhs
    matrices and ("V", i) square diagonal-block tiles stacked in an n x b
    matrix (the inverses of the diagonal factor tiles)."""
    tiles = (_Tile * max(1, len(names)))()
    for name, idx in names.items():
        m = mats[name[0]]
        n_rows, n_cols = m.shape
        if name[0] in ("X", "R", "D"):
            r0, c0 = name[1] * b, 0
            rows, cols = min(b, n_rows - r0), n_cols
        elif name[0] == "V":
            r0, c0 = name[1] * b, 0
            rows = cols = min(b, n_rows - r0)
        elif name[0] == "P":      # particle group: rows groups[i] .. groups[i+1]
            r0, c0 = int(groups[name[1]]), 0
            rows, cols = int(groups[name[1] + 1] - groups[name[1]]), n_cols
        else:
            r0, c0 = name[1] * b, name[2] * b
            rows, cols = min(b, n_rows - r0), min(b, n_cols - c0)
        ptr = m.ctypes.data + (r0 * m.strides[0] + c0 * m.strides[1])
        tiles[idx] = _Tile(ptr, rows, cols, m.strides[0] // 8, 0)
    return tiles


def execute(tasks, mats, b, groups=None):
    """Run a task list on numpy FP64 matrices in place, in insertion order.
    Returns the LAPACK-style info (0 = success)."""
    for m in mats.values():
        assert m.dtype == np.float64 and m.flags["C_CONTIGUOUS"]
    _, _, _, names = access_arrays(tasks)
    tiles = _tile_views(names, mats, b, groups)
    nt = len(tasks)
    ops = np.asarray([t[0] for t in tasks], np.int32)
    th = np.full((max(nt, 1), 4), -1, np.int32)
    for t, (_, acc, _) in enumerate(tasks):
        for s, (name, _) in enumerate(acc):
            th[t, s] = names[name]
    args = np.asarray([t[2] for t in tasks] or [0], np.int64)
    info = ctypes.c_int(0)
    rc = lib().spxo_execute(nt, _p(ops), _p(th), _p(args), ctypes.cast(tiles, ctypes.c_void_p),
                            len(names), ctypes.byref(info))
    if rc < 0:
        raise ValueError("malformed task list")
    return int(info.value)


def tiled_cholesky(A: np.ndarray, b: int, X: np.ndarray | None = None) -> int:
    """Tiled Cholesky of A in place (lower), optionally followed by the block
    solve of A Y = X in place.  Returns info."""
    n = A.shape[0]
    T = -(-n // b)
    mats = {"A": A}
    if X is not None:
        mats["X"] = X
    return execute(cholesky_tasks(T, b, with_solve=X is not None), mats, b)


def tiled_gemm(A, B, C, b, commutative=False):
    n = A.shape[0]
    T = -(-n // b)
    return execute(gemm_tasks(T, commutative), {"A": A, "B": B, "C": C}, b)


# ---------------------------------------------------------------------------
# Untiled references and metrics.
# ---------------------------------------------------------------------------

def potrf(A: np.ndarray) -> int:
    """Unblocked Cholesky-Crout of the whole matrix, in place (lower)."""
    assert A.dtype == np.float64 and A.flags["C_CONTIGUOUS"]
    return int(lib().spxo_potrf(_p(A), A.shape[0], A.shape[1]))


def solve_untiled(L: np.ndarray, X: np.ndarray) -> None:
    """Forward then back substitution with the lower factor L, X in place."""
    n, nrhs = X.shape
    lib().spxo_trsv_lower(_p(L), L.shape[1], _p(X), n, nrhs, nrhs)
    lib().spxo_trsv_lower_t(_p(L), L.shape[1], _p(X), n, nrhs, nrhs)


def gemm_untiled(A, B, C):
    lib().spxo_gemm_untiled(_p(A), _p(B), _p(C), A.shape[0])


def factor_backward_error(A: np.ndarray, L: np.ndarray) -> float:
    """||A - L L^T||_F / ||A||_F with compensated residuals (L = lower of L)."""
    return float(lib().spxo_factor_backward_error(_p(A), A.shape[1], _p(L), L.shape[1], A.shape[0]))


def solve_backward_error(A, X, B) -> np.ndarray:
    """Normwise backward error per column (Rigal-Gaches), compensated residual."""
    n, nrhs = X.shape
    eta = np.zeros(nrhs, np.float64)
    lib().spxo_solve_backward_error(_p(A), A.shape[1], _p(np.ascontiguousarray(X)),
                                    _p(np.ascontiguousarray(B)), n, nrhs, _p(eta))
    return eta


def freivalds(A, L, v) -> float:
    """||A v - L (L^T v)||_2 / (||A||_F ||v||_2), O(n^2)."""
    v = np.ascontiguousarray(v, np.float64)
    return float(lib().spxo_freivalds(_p(A), A.shape[1], _p(L), L.shape[1], A.shape[0], _p(v)))


def timed_tiled_cholesky(A: np.ndarray, b: int, X: np.ndarray | None = None):
    """Wall time (s) of the tiled oracle on one host core, and its info."""
    t0 = time.perf_counter()
    info = tiled_cholesky(A, b, X)
    return time.perf_counter() - t0, info
