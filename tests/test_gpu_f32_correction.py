"""GPU parity of the FP32 correction solve of mixed-precision refinement
(spx_solve_inv_f32_insert: FP64 residual rounded to FP32, the block solve
with the diagonal inverses on FP32 copies of the factor, the correction
added to the FP64 solution), against the oracle.

* sparse integer unit-lower factors: every intermediate is a small integer,
  exact in FP32, so x = 0 + (L L^T)^{-1} b equals the oracle's FP64 solve bit
  for bit;
* random factors: within FP32 rounding of the oracle's FP64 solve (normwise
  backward error <= 64 n 2^-24);
* refinement with the FP32 correction reaches the FP64 backward error bound
  in no more iterations (+1) than with the FP64 correction;
* operand rules: FP32 only for the narrow solve updates, no mixed types.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2308_15964_b300 import inputs
from tests._gpu import need_cuda, spx_mod
from tests.test_gpu_inverse import unit_lower

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    need_cuda()
    return spx_mod()


def gpu_f32_correction(S, L_np, R_np, b):
    """X = 0 + (L L^T)^{-1} R through the FP32 correction graph."""
    from paper_2308_15964_b300 import mixed
    n, nrhs = R_np.shape
    L = torch.from_numpy(np.ascontiguousarray(L_np)).cuda()
    V = torch.empty((n, min(b, n)), dtype=torch.float64, device="cuda")
    g = S.Graph()
    mixed.trtri_graph(g, L, b, V)
    assert g.run()[0] == 0
    g.close()
    L32 = torch.empty((n, n), dtype=torch.float32, device="cuda")
    V32 = torch.empty(V.shape, dtype=torch.float32, device="cuda")
    g = S.Graph()
    mixed.convert_graph(g, L, L32)
    mixed.convert_graph(g, V, V32)
    assert g.run()[0] == 0
    g.close()
    assert torch.equal(L32, L.float())
    R = torch.from_numpy(np.ascontiguousarray(R_np)).cuda()
    X = torch.zeros_like(R)
    R32 = torch.full(R.shape, float("nan"), dtype=torch.float32, device="cuda")
    D32 = torch.full(R.shape, float("nan"), dtype=torch.float32, device="cuda")
    g = S.Graph()
    mixed.solve_inv_f32_graph(g, L32, b, V32, R, R32, D32, X)
    assert g.run()[0] == 0
    g.close()
    return X.cpu().numpy()


def oracle_solve_inv(L, B, b):
    n = L.shape[0]
    T = -(-n // b)
    Ro, Do, Vo = B.copy(), np.zeros_like(B), np.zeros((n, b))
    assert O.execute(O.trtri_tasks(T), {"A": L, "V": Vo}, b) == 0
    assert O.execute(O.solve_inv_tasks(T), {"A": L, "V": Vo, "R": Ro, "D": Do}, b) == 0
    return Ro


@pytest.mark.parametrize("n,b,nrhs", [(300, 128, 1), (512, 128, 8), (200, 64, 16), (257, 64, 3)])
def test_f32_correction_integer_bit_exact(S, n, b, nrhs):
    L0 = unit_lower(n, 2 * n + b)
    x0 = np.random.default_rng(5).integers(-3, 4, size=(n, nrhs)).astype(np.float64)
    B = (L0 @ L0.T) @ x0
    # every intermediate of the solve is an integer of at most 2^24 in magnitude
    Linv = np.linalg.inv(L0)
    assert np.abs(np.rint(Linv) @ np.abs(B)).max() < 2.0 ** 24
    Xo = oracle_solve_inv(L0, B, b)
    assert np.array_equal(Xo, x0)
    assert np.array_equal(gpu_f32_correction(S, L0, B, b), Xo)


@pytest.mark.parametrize("n,b,nrhs", [(600, 128, 3), (1000, 256, 8), (777, 256, 16)])
def test_f32_correction_matches_oracle(S, n, b, nrhs):
    A = inputs.spd_matrix(n, 1.0, seed=n + 3).numpy()
    B = inputs.rhs(n, nrhs, seed=n + 3).numpy()
    L = A.copy()
    assert O.tiled_cholesky(L, b) == 0
    L = np.tril(L)
    Xo = oracle_solve_inv(L, B, b)
    Xg = gpu_f32_correction(S, L, B, b)
    assert O.solve_backward_error(A, Xg, B).max() <= 64 * n * 2.0 ** -24
    assert np.abs(Xg - Xo).max() <= 1e-3 * np.abs(Xo).max()


@pytest.mark.parametrize("prec,n,b,nrhs", [("tf32", 1536, 512, 3), ("tf32", 1000, 256, 8),
                                           ("bf16", 1536, 512, 3)])
def test_refinement_with_f32_correction(S, prec, n, b, nrhs):
    from paper_2308_15964_b300 import mixed
    p = S.TF32 if prec == "tf32" else S.BF16
    A = inputs.spd_matrix(n, 1e-2, seed=6)
    B = inputs.rhs(n, nrhs, seed=6)
    runs = {}
    for corr in ("f64", "f32"):
        X, _, info = mixed.mixed_solve(A.cuda(), B.cuda(), b=b, prec=p, correction=corr)
        assert info["status"] == 0
        runs[corr] = (X.cpu().numpy(), info)
    X, info = runs["f32"]
    assert info["converged"] == runs["f64"][1]["converged"]
    if info["converged"]:
        eta = O.solve_backward_error(A.numpy(), X, B.numpy()).max()
        assert eta <= 1e-14, eta
        assert abs(info["eta_final"] - eta) <= 1e-6 * eta
        assert info["iterations"] <= runs["f64"][1]["iterations"] + 1


def test_f32_operand_rules(S):
    n = 64
    keep = []    # tiles are keyed by address: keep every buffer alive

    def f32(*s):
        keep.append(torch.zeros(s, dtype=torch.float32, device="cuda"))
        return keep[-1]

    def f64(*s):
        keep.append(torch.zeros(s, dtype=torch.float64, device="cuda"))
        return keep[-1]

    g = S.Graph()
    L, Xk = g.register_tensor(f32(n, n), S.DT_F32), g.register_tensor(f32(n, 17), S.DT_F32)
    Xi = g.register_tensor(f32(n, 17), S.DT_F32)
    with pytest.raises(Exception):       # FP32 solve updates: at most 16 columns
        g.insert(S.OP_GEMM_FWD, [L, Xk, Xi], [S.READ, S.READ, S.WRITE])
    Yk, Yi = g.register_tensor(f32(n, 8), S.DT_F32), g.register_tensor(f64(n, 8))
    with pytest.raises(Exception):       # no mixed element types in one update
        g.insert(S.OP_GEMM_FWD, [L, Yk, Yi], [S.READ, S.READ, S.WRITE])
    L64 = g.register_tensor(f64(n, n))
    with pytest.raises(Exception):       # FP32 only where the op allows it
        g.insert(S.OP_POTRF, [g.register_tensor(f32(32, 32), S.DT_F32)], [S.WRITE])
    g.insert(S.OP_COPY, [L64, L], [S.READ, S.WRITE])        # FP64 -> FP32
    g.insert(S.OP_AXPY, [Yk, Yi], [S.READ, S.WRITE])        # FP32 -> FP64
    assert g.run()[0] == 0
    g.close()
    with pytest.raises(Exception):       # more than 16 right-hand sides
        from paper_2308_15964_b300 import mixed
        R = f64(n, 17)
        mixed.solve_inv_f32_graph(S.Graph(), f32(n, n), 32, f32(n, 32), R, f32(n, 17),
                                  f32(n, 17), f64(n, 17))
