"""GPU parity of the diagonal-tile inverses (TRTRI), the triangular products
(TRMM) and the block solve that applies the inverses, against the oracle.

* sparse integer unit-lower factors: inverses and solves are small exact
  integers, so the GPU results are bit-exact;
* random well-conditioned factors: within FP64 rounding of the oracle's
  substitution (different association, same arithmetic);
* narrow (<= 16 columns, 16-row units) and wide (64 x 64 units) right-hand
  sides, plain and transposed products, ragged last tiles.
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
    """Integer unit-lower matrix with about 1.5 entries of +-1 per row below
    the diagonal: its inverse stays a small-integer matrix (a dense one's
    entries grow exponentially with n and stop being exact in FP64)."""
    rng = np.random.default_rng(seed)
    L = np.eye(n)
    for i in range(1, n):
        k = rng.poisson(1.5)
        L[i, rng.integers(0, i, size=k)] = rng.choice([-1.0, 1.0], size=k)
    return L


def gpu_trtri(S, L_np, b):
    from paper_2308_15964_b300 import mixed
    n = L_np.shape[0]
    L = torch.from_numpy(np.ascontiguousarray(L_np)).cuda()
    V = torch.full((n, min(b, n)), float("nan"), dtype=torch.float64, device="cuda")
    g = S.Graph()
    mixed.trtri_graph(g, L, b, V)
    rc, _ = g.run()
    g.close()
    assert rc == 0
    return V.cpu().numpy()


def oracle_trtri(L_np, b):
    n = L_np.shape[0]
    V = np.zeros((n, min(b, n)))
    assert O.execute(O.trtri_tasks(-(-n // b)), {"A": np.ascontiguousarray(L_np), "V": V}, b) == 0
    return V


def blocks(V, n, b):
    """The square diagonal-tile inverses stored in V (the ragged last block
    covers only its own columns)."""
    out = []
    for k in range(-(-n // b)):
        r = slice(k * b, min(n, k * b + b))
        out.append(V[r, :r.stop - r.start])
    return out


@pytest.mark.parametrize("n,b", [(64, 64), (300, 128), (512, 512), (200, 64)])
def test_trtri_integer_bit_exact(S, n, b):
    L = unit_lower(n, n + b)
    for vg, vo in zip(blocks(gpu_trtri(S, L, b), n, b), blocks(oracle_trtri(L, b), n, b)):
        assert np.array_equal(vg, vo)


@pytest.mark.parametrize("n,b", [(300, 128), (512, 512), (130, 64)])
def test_trtri_matches_oracle(S, n, b):
    A = inputs.spd_matrix(n, 1.0, seed=n).numpy()
    L = np.tril(np.linalg.cholesky(A))
    for vg, vo in zip(blocks(gpu_trtri(S, L, b), n, b), blocks(oracle_trtri(L, b), n, b)):
        assert np.abs(vg - vo).max() <= 1e-13 * np.abs(vo).max()
        m = vg.shape[0]
        assert np.array_equal(np.triu(vg, 1), np.zeros((m, m)))  # zero above the diagonal


@pytest.mark.parametrize("nrhs", [1, 3, 8, 16, 40, 64])
@pytest.mark.parametrize("trans", [0, 1])
def test_trmm_matches_oracle(S, nrhs, trans):
    n = 200
    rng = np.random.default_rng(nrhs + 10 * trans)
    T = np.tril(rng.uniform(-1, 1, (n, n)))
    X = rng.uniform(-1, 1, (n, nrhs))
    Tg = torch.from_numpy(T).cuda()
    Xg = torch.from_numpy(X).cuda()
    Yg = torch.full((n, nrhs), float("nan"), dtype=torch.float64, device="cuda")
    g = S.Graph()
    t = g.insert(S.OP_TRMM, [g.register_tensor(Tg), g.register_tensor(Xg), g.register_tensor(Yg)],
                 [S.READ, S.READ, S.WRITE])
    g.set_arg(t, trans)
    rc, _ = g.run()
    g.close()
    assert rc == 0
    V, R, D = T.copy(), X.copy(), np.zeros_like(X)
    tasks = [(O.TRMM, [(("V", 0), O.READ), (("R", 0), O.READ), (("D", 0), O.WRITE)], trans)]
    assert O.execute(tasks, {"V": V, "R": R, "D": D}, n) == 0
    assert np.abs(Yg.cpu().numpy() - D).max() <= 1e-13 * max(1.0, np.abs(D).max())


def gpu_solve_inv(S, L_np, R_np, b):
    from paper_2308_15964_b300 import mixed
    n = L_np.shape[0]
    L = torch.from_numpy(np.ascontiguousarray(L_np)).cuda()
    V = torch.empty((n, min(b, n)), dtype=torch.float64, device="cuda")
    R = torch.from_numpy(np.ascontiguousarray(R_np)).cuda()
    D = torch.empty_like(R)
    g = S.Graph()
    mixed.trtri_graph(g, L, b, V)
    mixed.solve_inv_graph(g, L, b, V, R, D)
    rc, _ = g.run()
    g.close()
    assert rc == 0
    return R.cpu().numpy()


@pytest.mark.parametrize("n,b,nrhs", [(300, 128, 1), (512, 128, 8), (200, 64, 20)])
def test_solve_inv_integer_bit_exact(S, n, b, nrhs):
    L0 = unit_lower(n, 2 * n + b)
    x0 = np.random.default_rng(3).integers(-3, 4, size=(n, nrhs)).astype(np.float64)
    B = (L0 @ L0.T) @ x0
    assert np.array_equal(gpu_solve_inv(S, L0, B, b), x0)


@pytest.mark.parametrize("n,b,nrhs", [(600, 128, 3), (1000, 256, 8), (777, 256, 64)])
def test_solve_inv_matches_oracle(S, n, b, nrhs):
    A = inputs.spd_matrix(n, 1.0, seed=n + 1).numpy()
    B = inputs.rhs(n, nrhs, seed=n + 1).numpy()
    L = A.copy()
    assert O.tiled_cholesky(L, b) == 0
    L = np.tril(L)
    Xg = gpu_solve_inv(S, L, B, b)
    Ro, Do, Vo = B.copy(), np.zeros_like(B), np.zeros((n, b))
    T = -(-n // b)
    assert O.execute(O.trtri_tasks(T), {"A": L, "V": Vo}, b) == 0
    assert O.execute(O.solve_inv_tasks(T), {"A": L, "V": Vo, "R": Ro, "D": Do}, b) == 0
    assert np.abs(Xg - Ro).max() <= 1e-12 * np.abs(Ro).max()
    assert O.solve_backward_error(A, Xg, B).max() <= 1e-14


@pytest.mark.parametrize("inverse", [True, False])
def test_mixed_refinement_both_solves(S, inverse):
    from paper_2308_15964_b300 import mixed
    n = 2048
    A0 = inputs.spd_matrix(n, 1e-3, seed=8, device="cuda")
    B = inputs.rhs(n, 8, seed=8, device="cuda")
    X, L, info = mixed.mixed_solve(A0, B, b=512, prec=S.TF32, inverse=inverse)
    assert info["status"] == 0 and info["converged"]
    eta = O.solve_backward_error(A0.cpu().numpy(), X.cpu().numpy(), B.cpu().numpy())
    assert eta.max() <= 1e-14
