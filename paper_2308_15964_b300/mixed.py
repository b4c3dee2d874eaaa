"""Mixed-precision Cholesky solve with FP64 iterative refinement.

Factorization: one task graph (spx_cholesky_insert_mixed): POTRF on the
diagonal tiles in FP64, TRSM in FP64 writing a low-precision copy of each
factor tile, SYRK and GEMM trailing updates on the tensor cores (TF32 or
BF16 operands, FP32 accumulation) subtracted from the FP64 trailing matrix.
The first solve uses that factor.  Refinement (classical, on the host loop):
r = b - A x in FP64 with the normwise backward error of every right-hand side
computed on the device (spx_residual_eta_f64), L L^T d = r with the same
factor (a second, solve-only graph replayed through a CUDA graph; by default
it applies the FP64 inverses of the diagonal factor tiles, computed once by a
TRTRI graph, as products), x += d, until the backward error is <= tol or the
iteration cap is reached; non-convergence is reported, never hidden.

Stopping test: the fast plain FP64 residual drives the iterations; once its
eta is <= tol, a compensated residual (Dot2) recomputes eta, accurate to a
relative O(u), and only that value decides convergence.  If it is above tol,
or if the plain eta stops decreasing (its own rounding noise reached), every
later iteration uses the compensated residual, whose corrections also bring
x closer to the exact solution.  The host only compares the device's eta with
tol.
"""
from __future__ import annotations

import ctypes
import time

import torch

from . import spx

P = ctypes.c_void_p


def _p(t):
    return P(t.data_ptr())


def _s(stream):
    return P((stream or torch.cuda.current_stream()).cuda_stream)


def norm_inf(A, stream=None) -> torch.Tensor:
    out = torch.empty(1, dtype=torch.float64, device=A.device)
    spx._check(spx.lib.spx_norm_inf_f64(_p(A), A.shape[0], A.stride(0), _p(out), _s(stream)),
               "spx_norm_inf_f64")
    return out


def residual(A, X, B, R, norms, stream=None):
    n, nrhs = X.shape
    spx._check(spx.lib.spx_residual_f64(_p(A), n, A.stride(0), _p(X), X.stride(0), _p(B), B.stride(0),
                                        _p(R), R.stride(0), nrhs, _p(norms), _s(stream)),
               "spx_residual_f64")


def residual_eta(A, X, B, R, anorm, norms, eta, compensated=False, stream=None):
    """R = B - A X and eta[j] (normwise backward error per right-hand side),
    eta[nrhs] = max_j eta[j], all on the device; anorm = ||A||_inf (device)."""
    n, nrhs = X.shape
    spx._check(spx.lib.spx_residual_eta_f64(_p(A), n, A.stride(0), _p(X), X.stride(0), _p(B),
                                            B.stride(0), _p(R), R.stride(0), nrhs, _p(anorm),
                                            _p(norms), _p(eta), 1 if compensated else 0,
                                            _s(stream)),
               "spx_residual_eta_f64")


def axpy(Y, X, alpha=1.0, stream=None):
    spx._check(spx.lib.spx_axpy_f64(_p(Y), _p(X), Y.numel(), alpha, _s(stream)), "spx_axpy_f64")


def factor_graph(g: spx.Graph, A, Alo, b: int, X, prec: int, lookahead=True, V=None) -> int:
    """Insert the mixed-precision factorization (and the first solve when X is
    given).  With V (n x b FP64), the panel solves run as TRTRI into V plus
    TRSM_INV on the tensor cores (spx_cholesky_insert_mixed_inv); else as
    FP64 TRSM tasks."""
    n = A.shape[0]
    nt = ctypes.c_longlong()
    xa = (_p(X) if X is not None else None, X.shape[1] if X is not None else 0,
          X.stride(0) if X is not None else 0)
    if V is None:
        spx._check(spx.lib.spx_cholesky_insert_mixed(
            g._h, _p(A), n, A.stride(0), b, _p(Alo), Alo.stride(0), *xa,
            1 if lookahead else 0, prec, ctypes.byref(nt)), "spx_cholesky_insert_mixed")
    else:
        spx._check(spx.lib.spx_cholesky_insert_mixed_inv(
            g._h, _p(A), n, A.stride(0), b, _p(Alo), Alo.stride(0), _p(V), V.stride(0), *xa,
            1 if lookahead else 0, prec, ctypes.byref(nt)), "spx_cholesky_insert_mixed_inv")
        g._keep.append(V)
    g._keep.extend([A, Alo] + ([X] if X is not None else []))
    return nt.value


def solve_graph(g: spx.Graph, L, b: int, R) -> int:
    n = L.shape[0]
    nt = ctypes.c_longlong()
    spx._check(spx.lib.spx_solve_insert(g._h, _p(L), n, L.stride(0), b, _p(R), R.shape[1],
                                        R.stride(0), ctypes.byref(nt)), "spx_solve_insert")
    g._keep.extend([L, R])
    return nt.value


def trtri_graph(g: spx.Graph, L, b: int, V) -> int:
    """V (n x b) <- the inverses of the diagonal b x b tiles of L."""
    n = L.shape[0]
    nt = ctypes.c_longlong()
    spx._check(spx.lib.spx_trtri_insert(g._h, _p(L), n, L.stride(0), b, _p(V), V.stride(0),
                                        ctypes.byref(nt)), "spx_trtri_insert")
    g._keep.extend([L, V])
    return nt.value


def solve_inv_graph(g: spx.Graph, L, b: int, V, R, D) -> int:
    """Block solve L L^T x = r applying the diagonal inverses V: R in, R out,
    D scratch (same shape as R)."""
    n = L.shape[0]
    nt = ctypes.c_longlong()
    spx._check(spx.lib.spx_solve_inv_insert(g._h, _p(L), n, L.stride(0), b, _p(V), V.stride(0),
                                            _p(R), _p(D), R.shape[1], R.stride(0),
                                            ctypes.byref(nt)), "spx_solve_inv_insert")
    g._keep.extend([L, V, R, D])
    return nt.value


def convert_graph(g: spx.Graph, src, dst) -> int:
    """dst <- src (same shape; FP64 -> FP32 rounds to nearest) as one COPY task."""
    hs = g.register_tensor(src, _dt(src))
    hd = g.register_tensor(dst, _dt(dst))
    return g.insert(spx.OP_COPY, [hs, hd], [spx.READ, spx.WRITE])


def _dt(t):
    return spx.DT_F32 if t.dtype == torch.float32 else spx.DT_F64


def solve_inv_f32_graph(g: spx.Graph, L32, b: int, V32, R, R32, D32, X) -> int:
    """x <- x + (L L^T)^{-1} r with the solve in FP32 on the copies L32, V32:
    R (FP64 residual) in, X (FP64) updated, R32 / D32 FP32 scratch."""
    n, nrhs = R.shape
    nt = ctypes.c_longlong()
    spx._check(spx.lib.spx_solve_inv_f32_insert(g._h, _p(L32), n, L32.stride(0), b, _p(V32),
                                                V32.stride(0), _p(R), _p(R32), _p(D32), _p(X),
                                                nrhs, R.stride(0), ctypes.byref(nt)),
               "spx_solve_inv_f32_insert")
    return nt.value


def lowp_dtype(prec: int):
    return torch.bfloat16 if prec == spx.BF16 else torch.float32


def mixed_solve(A0, B, b: int = 512, prec: int = spx.TF32, tol: float = 1e-14,
                max_iter: int | None = None, inverse: bool = True, correction: str = "auto",
                panel: str = "tc"):
    """Solve A0 X = B.  Returns (X, L, info) where L holds the factor (lower
    triangle) and info has 'converged', 'iterations', 'eta' (history of the
    max normwise backward error, device-computed, plain or compensated
    residual per 'eta_compensated'), 'eta_final' (the last compensated eta:
    the certified backward error of the returned X), 'factor_ms',
    'refine_ms', 'status'.  With
    `inverse`, the correction solves apply the inverses of the diagonal factor
    tiles (computed once, FP64, timed in refine_ms) as products; otherwise
    they substitute.  `correction` = "f32" (with `inverse`, at most 16
    right-hand sides) solves for each correction in FP32 on FP32 copies of the
    factor and of the inverses: the factor is only accurate to TF32 / BF16, so
    FP32 costs the refinement no iterations and runs on the FP32 pipe; "f64"
    keeps the FP64 solve; "auto" (default) takes "f32" where it applies.
    `panel` = "tc" (default) runs the factorization's panel solves as TRTRI +
    TRSM_INV on the tensor cores (split TF32, about FP32 accuracy; the
    inverses then serve the correction solves too); "fp64" keeps FP64 TRSM
    tasks."""
    if max_iter is None:
        max_iter = 30 if prec == spx.TF32 else 50
    n, nrhs = B.shape
    if correction == "auto":
        correction = "f32" if inverse and nrhs <= 16 else "f64"
    if panel not in ("tc", "fp64"):
        raise ValueError("panel is 'tc' or 'fp64'")
    A = A0.clone()
    Alo = torch.zeros((n, n), dtype=lowp_dtype(prec), device=A0.device)
    X = B.clone()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    g = spx.Graph()
    V = (torch.empty((n, min(b, n)), dtype=torch.float64, device=A0.device)
         if panel == "tc" else None)
    factor_graph(g, A, Alo, b, X, prec, V=V)
    ev[0].record()
    rc, info = g.run()
    ev[1].record()
    st = g.stats()
    share = {k: v / max(1, st["total_cycles"]) for k, v in st["op_cycles"].items()}
    if rc != spx.OK:
        g.close()
        return X, A, {"status": rc, "info": info, "converged": False, "iterations": 0, "eta": []}
    R = torch.empty_like(B)
    gs = spx.Graph(cuda_graph=True)
    if inverse:
        D = torch.empty_like(B)
        if V is None:       # the factorization did not leave the inverses
            V = torch.empty((n, min(b, n)), dtype=torch.float64, device=A0.device)
            gt = spx.Graph()
            trtri_graph(gt, A, b, V)
            rc, _ = gt.run()
            gt.close()
            if rc != spx.OK:
                g.close()
                return X, A, {"status": rc, "converged": False, "iterations": 0, "eta": []}
        if correction == "f32":
            if nrhs > 16:
                raise ValueError("the FP32 correction solve takes at most 16 right-hand sides")
            L32 = torch.empty((n, n), dtype=torch.float32, device=A0.device)
            V32 = torch.empty(V.shape, dtype=torch.float32, device=A0.device)
            R32, D32 = (torch.empty(B.shape, dtype=torch.float32, device=A0.device)
                        for _ in range(2))
            gc = spx.Graph()
            convert_graph(gc, A, L32)
            convert_graph(gc, V, V32)
            rc, _ = gc.run()
            gc.close()
            if rc != spx.OK:
                g.close()
                return X, A, {"status": rc, "converged": False, "iterations": 0, "eta": []}
            solve_inv_f32_graph(gs, L32, b, V32, R, R32, D32, X)
        else:
            solve_inv_graph(gs, A, b, V, R, D)
    else:
        solve_graph(gs, A, b, R)
    anorm = norm_inf(A0)
    norms = torch.empty(3 * nrhs, dtype=torch.float64, device=A0.device)
    eta_d = torch.empty(nrhs + 1, dtype=torch.float64, device=A0.device)
    history, comp_flags = [], []
    converged = False
    compensated = False      # plain residuals until their eta reaches tol
    eta_final = None
    it = 0
    for it in range(max_iter + 1):
        residual_eta(A0, X, B, R, anorm, norms, eta_d, compensated)
        eta = float(eta_d[nrhs].item())
        history.append(eta)
        comp_flags.append(compensated)
        if compensated:
            eta_final = eta
            if eta <= tol:
                converged = True
                break
        elif eta <= tol or (len(history) > 1 and eta > 0.9 * history[-2]):
            # reached tol, or stagnated at the plain residual's rounding
            # noise: certify (and continue) with the compensated residual
            compensated = True
            residual_eta(A0, X, B, R, anorm, norms, eta_d, True)
            eta_final = float(eta_d[nrhs].item())
            history.append(eta_final)
            comp_flags.append(True)
            if eta_final <= tol:
                converged = True
                break
        if it == max_iter:
            break
        rc, _ = gs.run()
        if rc != spx.OK:
            break
        gs.reset()
        if not (inverse and correction == "f32"):   # the FP32 graph adds it itself
            axpy(X, R)
    ev[2].record()
    ev[2].synchronize()
    out = {"status": rc, "converged": converged, "iterations": it, "eta": history,
           "eta_compensated": comp_flags, "eta_final": eta_final,
           "factor_ms": ev[0].elapsed_time(ev[1]), "refine_ms": ev[1].elapsed_time(ev[2]),
           "factor_op_share": share, "correction": correction if inverse else "f64",
           "panel": panel}
    g.close()
    gs.close()
    return X, A, out


def gmres_ir_solve(A0, B, b: int = 512, prec: int = spx.BF16, tol: float = 1e-14,
                   max_outer: int = 20, max_inner: int = 30, inner_tol: float = 1e-10):
    """Solve A0 X = B with the mixed-precision factor (tensor-core panel and
    trailing updates, FP64 POTRF) and GMRES-based refinement (spx_gmres_ir):
    each refinement step solves the correction equation by FP64 GMRES
    preconditioned with the factor (its solve graph applying the FP64
    inverses of the diagonal tiles).  Returns (X, L, info) with 'converged',
    'outer', 'inner', 'eta_final' (certified when converged), 'factor_ms',
    'refine_ms', 'status'."""
    n, nrhs = B.shape
    A = A0.clone()
    Alo = torch.zeros((n, n), dtype=lowp_dtype(prec), device=A0.device)
    X = B.clone()
    V = torch.empty((n, min(b, n)), dtype=torch.float64, device=A0.device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    g = spx.Graph()
    factor_graph(g, A, Alo, b, X, prec, V=V)
    ev[0].record()
    rc, info = g.run()
    ev[1].record()
    g.close()
    if rc != spx.OK:
        return X, A, {"status": rc, "info": info, "converged": False, "outer": 0, "inner": 0}
    R, D = torch.empty_like(B), torch.empty_like(B)
    gp = spx.Graph(cuda_graph=True)
    solve_inv_graph(gp, A, b, V, R, D)
    wbytes = spx.lib.spx_gmres_ir_workspace(n, nrhs, max_inner)
    if wbytes < 0:
        raise ValueError("unsupported GMRES size")
    work = torch.empty(wbytes // 8 + 1, dtype=torch.float64, device=A0.device)
    cfg = spx.GmresConfig(max_outer, max_inner, inner_tol, tol)
    res = spx.GmresResult()
    rc = spx.lib.spx_gmres_ir(_p(A0), n, A0.stride(0), _p(B), _p(X), nrhs, gp._h, _p(R), _p(work),
                              wbytes, ctypes.byref(cfg), ctypes.byref(res), _s(None))
    ev[2].record()
    ev[2].synchronize()
    gp.close()
    spx._check(rc, "spx_gmres_ir")
    return X, A, {"status": rc, "converged": bool(res.converged), "outer": res.outer,
                  "inner": res.inner, "eta_final": res.eta,
                  "factor_ms": ev[0].elapsed_time(ev[1]), "refine_ms": ev[1].elapsed_time(ev[2])}
