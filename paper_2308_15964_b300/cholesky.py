"""Task graphs of the paper's workloads, inserted through the C ABI.

* tiled Cholesky (section "Numerical applications": POTRF on diagonal tiles,
  TRSM, SYRK and GEMM on the others), right-looking, k outer, followed by the
  block forward and back solves of A X = B (spx_cholesky_insert);
* tiled GEMM C += A B with one task per (i, j, k) depending on the block C_ij
  (spx_gemm_insert).

Matrices are row-major FP64 torch CUDA tensors (or raw device pointers).  The
graph refers to their memory; the caller keeps them alive until the graph has
been waited for.
"""
from __future__ import annotations

import ctypes

from . import spx


def _ptr(t):
    return ctypes.c_void_p(t if isinstance(t, int) else t.data_ptr())


def cholesky_graph(g: spx.Graph, A, b: int, X=None, lookahead: bool = True, prec: int = spx.F64):
    """Insert A = L L^T (lower, in place) and, when X is given, the solve
    A Y = X (Y written over X).  Returns the number of tasks inserted."""
    n = A.shape[0]
    assert A.stride(1) == 1 and (X is None or X.stride(1) == 1)
    nt = ctypes.c_longlong()
    spx._check(spx.lib.spx_cholesky_insert(
        g._h, _ptr(A), n, A.stride(0), b, _ptr(X) if X is not None else None,
        X.shape[1] if X is not None else 0, X.stride(0) if X is not None else 0,
        int(lookahead), prec, ctypes.byref(nt)), "spx_cholesky_insert")
    g._keep.extend([A] + ([X] if X is not None else []))
    return nt.value


def ozaki_store(n: int, b: int, device="cuda", inverse_panels: bool = False):
    """The split store of spx_cholesky_insert_ozaki for an n x n matrix in
    b x b tiles: T (T - 1) / 2 slots (T more with inverse panels) of
    spx_ozaki_slot_bytes(b) bytes (torch allocations are 256-byte aligned)."""
    import torch
    T = -(-n // b)
    slot = spx.lib.spx_ozaki_slot_bytes(b)
    if slot <= 0:
        raise ValueError(f"tile {b}: the split path takes b a multiple of 32 in [32, 512]")
    nslots = T * (T - 1) // 2 + (T if inverse_panels else 0)
    return torch.empty(max(1, nslots) * slot, dtype=torch.uint8, device=device)


def cholesky_ozaki_graph(g: spx.Graph, A, b: int, X=None, lookahead: bool = True, S=None,
                         V=None, fuse_panel: bool = False):
    """spx_cholesky_insert_ozaki: A = L L^T with the trailing updates in FP64
    emulated on the tensor cores (digit planes in the split store S, made by
    ozaki_store when None).  V (n x b FP64, or None): inverse panels, V
    receiving the inverses of the diagonal factor tiles.  Returns the number
    of tasks inserted.  fuse_panel: POTRF and the critical panel tile's solve as
    one POTRF_PANEL task."""
    n = A.shape[0]
    assert A.stride(1) == 1 and (X is None or X.stride(1) == 1)
    assert V is None or (V.stride(1) == 1 and V.shape[0] >= n)
    if S is None:
        S = ozaki_store(n, b, A.device, inverse_panels=V is not None)
    nt = ctypes.c_longlong()
    spx._check(spx.lib.spx_cholesky_insert_ozaki(
        g._h, _ptr(A), n, A.stride(0), b, _ptr(S), S.numel() * S.element_size(),
        _ptr(V) if V is not None else None, V.stride(0) if V is not None else 0,
        1 if fuse_panel else 0, _ptr(X) if X is not None else None, X.shape[1] if X is not None else 0,
        X.stride(0) if X is not None else 0, int(lookahead), ctypes.byref(nt)),
        "spx_cholesky_insert_ozaki")
    g._keep.extend([A, S] + ([X] if X is not None else []) + ([V] if V is not None else []))
    return nt.value


def cholesky_host_ozaki(g: spx.Graph, A_host, L_host, b: int, dev_A=None, S=None, V=None,
                        stream=None):
    """spx_cholesky_host_ozaki: the split-path Cholesky (inverse panels) of the
    host matrix A_host (pinned CPU float64 tensor, row-major), its factor in
    L_host's lower triangle; the column blocks are uploaded while the kernel
    runs.  Device buffers are allocated when not given.  Returns (status,
    info): spx.OK, or spx.NOT_SPD with the failed column."""
    import torch
    n = A_host.shape[0]
    assert A_host.stride(1) == 1 and L_host.stride(0) == A_host.stride(0) and L_host.stride(1) == 1
    if dev_A is None:
        dev_A = torch.empty((n, n), dtype=torch.float64, device="cuda")
    if S is None:
        S = ozaki_store(n, b, dev_A.device, inverse_panels=True)
    if V is None:
        V = torch.empty((n, min(b, n)), dtype=torch.float64, device=dev_A.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    info = ctypes.c_int()
    rc = spx.lib.spx_cholesky_host_ozaki(
        g._h, _ptr(A_host), _ptr(L_host), n, A_host.stride(0), b, _ptr(dev_A), dev_A.stride(0),
        _ptr(S), S.numel() * S.element_size(), _ptr(V), V.stride(0),
        ctypes.c_void_p(st.cuda_stream), ctypes.byref(info))
    if rc not in (spx.OK, spx.NOT_SPD):
        spx._check(rc, "spx_cholesky_host_ozaki")
    g._keep.extend([dev_A, S, V])
    return rc, info.value


def gemm_graph(g: spx.Graph, A, B, C, b: int, commutative: bool = False, atomic: bool = False):
    """Insert C += A B, one task per (i, j, k), i and j outer, k inner, with a
    WRITE, COMMUTATIVE_WRITE (commutative) or ATOMIC_WRITE (atomic) on C_ij."""
    n = A.shape[0]
    assert A.stride(0) == B.stride(0) == C.stride(0)
    nt = ctypes.c_longlong()
    sel = 2 if atomic else (1 if commutative else 0)
    spx._check(spx.lib.spx_gemm_insert(g._h, _ptr(A), _ptr(B), _ptr(C), n, A.stride(0), b,
                                       sel, ctypes.byref(nt)), "spx_gemm_insert")
    g._keep.extend([A, B, C])
    return nt.value


def gemm_ozaki_graph(g: spx.Graph, A, B, C, b: int, commutative: bool = False, S=None):
    """spx_gemm_insert_ozaki: C += A B with the products in FP64 emulated on
    the tensor cores: SPLIT tasks for the tiles of A, SPLIT_T for those of B,
    then one GEMM_NN_ADD per (i, j, k) (WRITE, or COMMUTATIVE_WRITE on C_ij).
    S: the split store (2 T^2 slots; allocated when None).  Returns the
    number of tasks inserted."""
    import torch
    n = A.shape[0]
    assert A.stride(0) == B.stride(0) == C.stride(0) and A.stride(1) == 1
    T = -(-n // b)
    slot = spx.lib.spx_ozaki_slot_bytes(b)
    if slot <= 0:
        raise ValueError(f"tile {b}: the split path takes b a multiple of 32 in [32, 512]")
    if S is None:
        S = torch.empty(2 * T * T * slot, dtype=torch.uint8, device=A.device)
    nt = ctypes.c_longlong()
    spx._check(spx.lib.spx_gemm_insert_ozaki(g._h, _ptr(A), _ptr(B), _ptr(C), n, A.stride(0), b,
                                             1 if commutative else 0, _ptr(S),
                                             S.numel() * S.element_size(), ctypes.byref(nt)),
               "spx_gemm_insert_ozaki")
    g._keep.extend([A, B, C, S])
    return nt.value


def cholesky_flops(n: int, nrhs: int = 0) -> float:
    """Algorithmic flops: n^3/3 for the factorization (leading order, exact
    for the tiled task counts) plus 2 n^2 per right-hand side for the solve."""
    return n ** 3 / 3.0 + 2.0 * n * n * nrhs


def gemm_flops(n: int) -> float:
    return 2.0 * n ** 3
