"""The mixed-precision panel solve on the tensor cores (TRSM_INV: A_ik <-
A_ik V_k^T with V_k = L_kk^{-1} from TRTRI, split-TF32 products) against the
oracle.

* the op alone: within the split-TF32 error bound of the oracle's FP64
  product, ragged rows and a 64-wide last column block included; the
  low-precision copy is exactly the TF32 / BF16 rounding of the FP64 result;
* an integer pin: A = L0 L0^T with L0 unit lower, diagonal tiles I - S (S the
  ones below the diagonal, so every V_k holds only 0 and 1) and off-diagonal
  entries in {-1, 0, 1}: every operand, product and partial sum is an exact
  small integer, so factor and solve are bit-exact, also with a ragged last
  tile;
* refinement from that factor reaches eta <= 1e-14 by the oracle, at the
  conditioning of the large mixed-precision workload (sigma = 1e-3) too, in
  at most two more iterations than with the FP64 panel solve.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2308_15964_b300 import inputs
from tests._gpu import need_cuda, spx_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    need_cuda()
    return spx_mod()


def tf32_rna(x32: np.ndarray) -> np.ndarray:
    """FP32 -> TF32 (nearest, ties away from zero), kept in FP32 storage."""
    u = x32.astype(np.float32).view(np.uint32)
    return ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("m,n", [(512, 512), (200, 320), (128, 96), (77, 64)])
def test_trsm_inv_op_vs_oracle(S, prec, m, n):
    from paper_2308_15964_b300 import mixed
    p = S.TF32 if prec == "tf32" else S.BF16
    Lkk = inputs.spd_matrix(n, 1.0, seed=m + n).numpy()
    assert O.potrf(Lkk) == 0
    Lkk = np.tril(Lkk)
    V = O.trtri(Lkk)
    A = inputs.uniform((m, n), m * n).numpy()
    ref = A.copy()
    mats = {"V": V.copy(), "A": ref}
    # one TRSM_INV task on the oracle (tile names: V block 0, A block (0, 0))
    info = O.execute([(O.TRSM_INV, [(("V", 0), O.READ), (("A", 0, 0), O.WRITE)], 0)], mats,
                     max(m, n))
    assert info == 0
    Vd = torch.from_numpy(V).cuda()
    Ad = torch.from_numpy(A.copy()).cuda()
    lo = torch.zeros((m, n), dtype=mixed.lowp_dtype(p), device="cuda")
    g = S.Graph()
    S.lib.spx_lowp_register(g._h, S.ctypes.c_void_p(lo.data_ptr()), m, n, n,
                            S.DT_BF16 if prec == "bf16" else S.DT_F32, None)
    hv = g.register_tensor(Vd)
    ha = g.register(Ad.data_ptr(), m, n, n, S.DT_F64, lo.data_ptr(), n)
    g.insert(S.OP_TRSM_INV, [hv, ha], [S.READ, S.WRITE], prec=p)
    assert g.run()[0] == 0
    torch.cuda.synchronize()
    got = Ad.cpu().numpy()
    # split TF32: |x - hi - lo| <= 1.25 2^-22 |x| per operand, the dropped
    # lo*lo term, and FP32 accumulation over n terms
    scale = np.abs(A) @ np.abs(V).T
    bound = (4 * 2.0 ** -22 + n * 2.0 ** -24) * scale
    assert (np.abs(got - ref) <= bound).all(), np.max(np.abs(got - ref) / scale)
    got32 = got.astype(np.float32)
    assert np.array_equal(got32.astype(np.float64), got)    # FP32 values, widened exactly
    if prec == "tf32":
        assert np.array_equal(lo.cpu().numpy(), tf32_rna(got32))
    else:
        assert torch.equal(lo.cpu(), torch.from_numpy(got32).to(torch.bfloat16))
    g.close()


def bidiag_lower(n, b, seed):
    """L0: unit lower; diagonal tiles I - S, entries of the off-diagonal
    tiles in {-1, 0, 1}."""
    rng = np.random.default_rng(seed)
    L = np.tril(rng.integers(-1, 2, size=(n, n)).astype(np.float64), -1)
    for k in range(0, n, b):
        e = min(n, k + b)
        L[k:e, k:e] = np.eye(e - k) - np.eye(e - k, k=-1)
    return L


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("n,b", [(1024, 256), (1000, 256), (640, 128)])
def test_integer_factor_bit_exact_inv(S, prec, n, b):
    from paper_2308_15964_b300 import mixed
    p = S.TF32 if prec == "tf32" else S.BF16
    L0 = bidiag_lower(n, b, n + b)
    A = L0 @ L0.T
    x0 = np.random.default_rng(3).integers(-3, 4, size=(n, 2)).astype(np.float64)
    Ad = torch.from_numpy(A).cuda()
    Xd = torch.from_numpy(A @ x0).cuda()
    Alo = torch.zeros((n, n), dtype=mixed.lowp_dtype(p), device="cuda")
    V = torch.zeros((n, b), dtype=torch.float64, device="cuda")
    outs = []
    for ex in (S.EXEC_PERSISTENT, S.EXEC_PER_TASK):
        A1, X1 = Ad.clone(), Xd.clone()
        g = S.Graph(executor=ex)
        mixed.factor_graph(g, A1, Alo, b, X1, p, V=V)
        rc, _ = g.run()
        assert rc == 0
        g.close()
        assert np.array_equal(np.tril(A1.cpu().numpy()), L0)
        assert np.array_equal(X1.cpu().numpy(), x0)
        outs.append(A1)
    assert torch.equal(outs[0], outs[1])
    # V holds the inverses of the diagonal tiles: lower triangles of ones
    Vh = V.cpu().numpy()
    for k in range(0, n, b):
        bk = min(b, n - k)
        assert np.array_equal(Vh[k:k + bk, :bk], np.tril(np.ones((bk, bk))))


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("n,sigma", [(1536, 1e-2), (2048, 1e-3), (4096, 1e-3)])
def test_refinement_with_tc_panel(S, prec, n, sigma):
    from paper_2308_15964_b300 import mixed
    p = S.TF32 if prec == "tf32" else S.BF16
    A = inputs.spd_matrix(n, sigma, seed=7)
    B = inputs.rhs(n, 8, seed=7)
    runs = {}
    for panel in ("fp64", "tc"):
        X, L, info = mixed.mixed_solve(A.cuda(), B.cuda(), b=512, prec=p, panel=panel)
        assert info["status"] == 0
        runs[panel] = (X.cpu().numpy(), L, info)
    X, L, info = runs["tc"]
    eta = O.solve_backward_error(A.numpy(), X, B.numpy())
    assert abs(info["eta_final"] - eta.max()) <= 1e-6 * eta.max()
    print(f"tc panel n={n} sigma={sigma} {prec}: converged={info['converged']} "
          f"iterations={info['iterations']} (fp64 panel {runs['fp64'][2]['iterations']}) "
          f"eta={eta.max():.3e}")
    if runs["fp64"][2]["converged"]:
        assert info["converged"], info["eta"]
        assert eta.max() <= 1e-14
        assert info["iterations"] <= runs["fp64"][2]["iterations"] + 2
    if not info["converged"]:
        assert info["iterations"] == (30 if p == S.TF32 else 50)
    beta = O.factor_backward_error(A.numpy(), L.cpu().numpy())
    assert beta < (2e-3 if p == S.TF32 else 2e-2), beta
