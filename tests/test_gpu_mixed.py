"""GPU parity of the mixed-precision Cholesky (tensor-core TF32 / BF16
trailing updates, FP64 POTRF) and of FP64 iterative refinement.

* integer unit-lower factors: every product and partial sum is an exact
  integer in BF16/TF32 operands with FP32 accumulation, so the factor and the
  solve are bit-exact on the mixed path too;
* random SPD systems: refinement reaches the FP64 normwise backward error
  <= 1e-14 (recomputed by the oracle with compensated residuals), or reports
  non-convergence with its iteration count, also at sigma = 1e-3 (condition
  number ~1e3, the conditioning of the large mixed-precision workload);
* the device's own backward error (compensated residual, the stopping test)
  equals the oracle's to a relative 1e-6, and on a hand-worked 3 x 3 case
  equals the closed form exactly;
* executors agree bit for bit.
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


def unit_lower(n, seed):
    rng = np.random.default_rng(seed)
    L = np.tril(rng.integers(-1, 2, size=(n, n)).astype(np.float64), -1)
    np.fill_diagonal(L, 1.0)
    return L


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("n,b", [(1024, 256), (1000, 256), (768, 384)])
def test_integer_factor_bit_exact(S, prec, n, b):
    from paper_2308_15964_b300 import mixed
    p = S.TF32 if prec == "tf32" else S.BF16
    L0 = unit_lower(n, n + b)
    A = L0 @ L0.T
    x0 = np.random.default_rng(2).integers(-3, 4, size=(n, 2)).astype(np.float64)
    Ad = torch.from_numpy(A).cuda()
    Xd = torch.from_numpy(A @ x0).cuda()
    Alo = torch.zeros((n, n), dtype=mixed.lowp_dtype(p), device="cuda")
    outs = []
    for ex in (S.EXEC_PERSISTENT, S.EXEC_PER_TASK, S.EXEC_STREAMS):
        A1, X1 = Ad.clone(), Xd.clone()
        g = S.Graph(executor=ex)
        mixed.factor_graph(g, A1, Alo, b, X1, p)
        rc, _ = g.run()
        assert rc == 0
        g.close()
        assert np.array_equal(np.tril(A1.cpu().numpy()), L0)
        assert np.array_equal(X1.cpu().numpy(), x0)
        outs.append(A1)
    assert all(torch.equal(outs[0], o) for o in outs[1:])


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_refinement_reaches_fp64(S, prec):
    from paper_2308_15964_b300 import mixed
    p = S.TF32 if prec == "tf32" else S.BF16
    n, b, nrhs = 1536, 512, 3
    A = inputs.spd_matrix(n, 1e-2, seed=4)
    B = inputs.rhs(n, nrhs, seed=4)
    X, L, info = mixed.mixed_solve(A.cuda(), B.cuda(), b=b, prec=p)
    assert info["status"] == 0
    eta = O.solve_backward_error(A.numpy(), X.cpu().numpy(), B.numpy())
    if info["converged"]:
        assert eta.max() <= 1e-14, (eta, info["eta"])
    else:
        assert info["iterations"] == (30 if p == S.TF32 else 50)
    # the device's certified eta is the oracle's, to rounding
    assert abs(info["eta_final"] - eta.max()) <= 1e-6 * eta.max(), (info["eta_final"], eta)
    if p == S.TF32:
        assert info["converged"], info["eta"]
    # the low-precision factor itself: backward error of order the precision
    beta = O.factor_backward_error(A.numpy(), L.cpu().numpy())
    assert beta < (2e-3 if p == S.TF32 else 2e-2), beta


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("n", [2048, 4096])
def test_refinement_sigma_1e3(S, prec, n):
    """A = B B^T/n + 1e-3 I (condition number ~1.3e3, as in the n = 32768
    mixed-precision workload), tile 512, 8 right-hand sides.  TF32 must
    converge to eta <= 1e-14 by the oracle.  BF16 (unit roundoff 2^-8, so
    kappa u > 1) may not: then its iteration count is the cap and its last
    eta is reported, never a claimed convergence."""
    from paper_2308_15964_b300 import mixed
    p = S.TF32 if prec == "tf32" else S.BF16
    A = inputs.spd_matrix(n, 1e-3, seed=4)
    B = inputs.rhs(n, 8, seed=4)
    X, L, info = mixed.mixed_solve(A.cuda(), B.cuda(), b=512, prec=p)
    assert info["status"] == 0
    eta = O.solve_backward_error(A.numpy(), X.cpu().numpy(), B.numpy())
    assert abs(info["eta_final"] - eta.max()) <= 1e-6 * eta.max(), (info["eta_final"], eta)
    print(f"sigma=1e-3 n={n} {prec}: converged={info['converged']} "
          f"iterations={info['iterations']} eta(oracle)={eta.max():.3e}")
    if info["converged"]:
        assert eta.max() <= 1e-14, (eta, info["eta"])
    else:
        assert info["iterations"] == (30 if p == S.TF32 else 50)
        assert info["eta_final"] > 1e-14
    if p == S.TF32:
        assert info["converged"], info["eta"]


def test_residual_eta_closed_form(S):
    """The hand-worked 3 x 3 case of the oracle's pin: eta = (1/44, 1/109)
    exactly (||A||_inf = 5, residuals 1/2 and 1/4, ||x||_inf = 3, ||b||_inf =
    7 and 49/4), with the plain and the compensated residual."""
    from paper_2308_15964_b300 import mixed
    A = torch.tensor([[4.0, -1.0, 0.0], [1.0, 3.0, 1.0], [0.0, -2.0, 1.0]],
                     dtype=torch.float64, device="cuda")
    X = torch.tensor([[1.0, -3.0], [-2.0, 0.0], [3.0, 1.0]], dtype=torch.float64, device="cuda")
    B = torch.tensor([[6.0, -12.25], [-1.5, -2.0], [7.0, 1.125]], dtype=torch.float64,
                     device="cuda")
    R = torch.empty_like(B)
    norms = torch.empty(6, dtype=torch.float64, device="cuda")
    eta = torch.empty(3, dtype=torch.float64, device="cuda")
    anorm = mixed.norm_inf(A)
    for comp in (False, True):
        mixed.residual_eta(A, X, B, R, anorm, norms, eta, compensated=comp)
        e = eta.cpu().numpy()
        assert e[0] == 1.0 / 44.0 and e[1] == 1.0 / 109.0 and e[2] == 1.0 / 44.0, e
        assert np.array_equal(R.cpu().numpy(), [[0.0, -0.25], [0.5, 0.0], [0.0, 0.125]])


@pytest.mark.parametrize("n,nrhs", [(700, 5), (1500, 8), (333, 16), (257, 1)])
def test_compensated_eta_vs_oracle(S, n, nrhs):
    """At a converged solution (the oracle's FP64 solve) the residual is pure
    rounding: the compensated device eta equals the oracle's (also
    compensated) to a relative 1e-6; the plain one only to gamma_n."""
    from paper_2308_15964_b300 import mixed
    A = inputs.spd_matrix(n, 1e-2, seed=n).numpy()
    B = inputs.rhs(n, nrhs, seed=n).numpy()
    L, X = A.copy(), B.copy()
    assert O.tiled_cholesky(L, 64, X) == 0
    ref = O.solve_backward_error(A, X, B)
    Ad, Xd, Bd = (torch.from_numpy(np.ascontiguousarray(v)).cuda() for v in (A, X, B))
    R = torch.empty_like(Bd)
    norms = torch.empty(3 * nrhs, dtype=torch.float64, device="cuda")
    eta = torch.empty(nrhs + 1, dtype=torch.float64, device="cuda")
    anorm = mixed.norm_inf(Ad)
    mixed.residual_eta(Ad, Xd, Bd, R, anorm, norms, eta, compensated=True)
    e = eta.cpu().numpy()
    assert np.all(np.abs(e[:nrhs] - ref) <= 1e-6 * ref), (e, ref)
    assert e[nrhs] == e[:nrhs].max()
    mixed.residual_eta(Ad, Xd, Bd, R, anorm, norms, eta, compensated=False)
    e = eta.cpu().numpy()
    assert np.all(np.abs(e[:nrhs] - ref) <= n * 1.2e-16), (e, ref)


def test_residual_kernel_vs_oracle(S):
    from paper_2308_15964_b300 import mixed
    n, nrhs = 700, 5
    A = inputs.spd_matrix(n, 1.0, seed=8)
    X = inputs.uniform((n, nrhs), 9)
    B = inputs.uniform((n, nrhs), 10)
    Ad, Xd, Bd = A.cuda(), X.cuda(), B.cuda()
    R = torch.empty_like(Bd)
    norms = torch.empty(3 * nrhs, dtype=torch.float64, device="cuda")
    mixed.residual(Ad, Xd, Bd, R, norms)
    ref = B.numpy() - A.numpy() @ X.numpy()
    scale = np.abs(A.numpy()) @ np.abs(X.numpy()) + np.abs(B.numpy())
    assert (np.abs(R.cpu().numpy() - ref) <= n * 2.2e-16 * scale).all()
    nv = norms.cpu().numpy()
    assert np.allclose(nv[:nrhs], np.abs(R.cpu().numpy()).max(0))
    assert np.array_equal(nv[nrhs:2 * nrhs], np.abs(X.numpy()).max(0))
    assert np.array_equal(nv[2 * nrhs:], np.abs(B.numpy()).max(0))
    an = mixed.norm_inf(Ad).item()
    assert abs(an - np.abs(A.numpy()).sum(1).max()) <= 1e-12 * an


def test_refinement_sweeps_as_tasks(S):
    """Refinement sweeps inserted as graph tasks (COPY, GEMM_FWD with the
    original matrix, block solves, AXPY) after the mixed factorization."""
    import ctypes
    from paper_2308_15964_b300 import mixed
    n, b, nrhs = 1024, 256, 3
    A = inputs.spd_matrix(n, 1.0, seed=12)
    B = inputs.rhs(n, nrhs, seed=12)
    Ad, A0, Bd = A.cuda(), A.cuda(), B.cuda()
    X, R = Bd.clone(), torch.empty_like(Bd)
    Alo = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    g = S.Graph()
    mixed.factor_graph(g, Ad, Alo, b, X, S.TF32)
    P = ctypes.c_void_p
    nt = ctypes.c_longlong()
    assert S.lib.spx_refine_insert(g._h, P(A0.data_ptr()), n, n, P(Ad.data_ptr()), n, b,
                                   P(Bd.data_ptr()), P(X.data_ptr()), P(R.data_ptr()), nrhs, nrhs, 4,
                                   ctypes.byref(nt)) == 0
    rc, _ = g.run()
    assert rc == 0
    eta = O.solve_backward_error(A.numpy(), X.cpu().numpy(), B.numpy())
    assert eta.max() <= 1e-14, eta
    g.close()


@pytest.mark.parametrize("n,b,nrhs", [(1024, 256, 3), (1000, 256, 8)])
def test_refinement_sweeps_with_inverses(S, n, b, nrhs):
    """The same in-graph sweeps with the correction solves applying the FP64
    inverses of the diagonal tiles (TRTRI tasks, then TRMM products): the
    backward error reaches the FP64 bound, and the result agrees with the
    substitution form to rounding."""
    import ctypes
    from paper_2308_15964_b300 import mixed
    A = inputs.spd_matrix(n, 1.0, seed=13)
    B = inputs.rhs(n, nrhs, seed=13)
    P = ctypes.c_void_p
    out = []
    for inverse in (True, False):
        Ad, A0, Bd = A.cuda(), A.cuda(), B.cuda()
        X, R, D = Bd.clone(), torch.empty_like(Bd), torch.empty_like(Bd)
        V = torch.empty((n, b), dtype=torch.float64, device="cuda")
        Alo = torch.zeros((n, n), dtype=torch.float32, device="cuda")
        g = S.Graph()
        mixed.factor_graph(g, Ad, Alo, b, X, S.TF32)
        nt = ctypes.c_longlong()
        if inverse:
            rc = S.lib.spx_refine_inv_insert(g._h, P(A0.data_ptr()), n, n, P(Ad.data_ptr()), n, b,
                                             P(V.data_ptr()), b, P(Bd.data_ptr()), P(X.data_ptr()),
                                             P(R.data_ptr()), P(D.data_ptr()), nrhs, nrhs, 4,
                                             ctypes.byref(nt))
        else:
            rc = S.lib.spx_refine_insert(g._h, P(A0.data_ptr()), n, n, P(Ad.data_ptr()), n, b,
                                         P(Bd.data_ptr()), P(X.data_ptr()), P(R.data_ptr()), nrhs,
                                         nrhs, 4, ctypes.byref(nt))
        assert rc == 0
        rc, _ = g.run()
        assert rc == 0
        g.close()
        x = X.cpu().numpy()
        assert O.solve_backward_error(A.numpy(), x, B.numpy()).max() <= 1e-14
        out.append(x)
    assert np.abs(out[0] - out[1]).max() <= 1e-11 * np.abs(out[1]).max()
