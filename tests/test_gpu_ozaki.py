"""FP64 trailing updates emulated on the tensor cores (prec SPX_F64_OZAKI)
against the oracle.

* op level, bit for bit against the oracle's split product (oracle/ozaki.py):
  a TRSM with an identity diagonal tile leaves its tile unchanged and splits
  it, so its digit planes and row exponents must equal the oracle's split;
  GEMM_NT_SUB and SYRK must then equal the oracle's gemm_nt_sub / syrk_lower
  exactly: rows of spread magnitudes, zero rows, ragged shapes and K, and the
  worst case of the digit sums (P_7 just below 2^24), which the tensor cores
  must accumulate exactly;
* the whole factorization + solve against the FP64 oracle with the FP64
  path's tolerances (entry error <= 1e-12, backward errors <= 1e-14); the
  integer and diagonal pins bit for bit; non-SPD info; bit-identical across
  runs and executors.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import ozaki as Z
from paper_2308_15964_b300 import inputs
from tests._gpu import need_cuda, spx_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    need_cuda()
    return spx_mod()


def r32(x):
    return (x + 31) // 32 * 32


def slot_view(store, slot_bytes, i, b):
    """(planes [8, b, b] float32, exponents [b] int32) of slot i."""
    raw = store[i * slot_bytes:(i + 1) * slot_bytes]
    # plane, 16-digit K chunk, row, digit -> plane, row, column
    planes = (raw[:16 * b * b].view(torch.bfloat16).float().reshape(8, b // 16, b, 16)
              .permute(0, 2, 1, 3).reshape(8, b, b).cpu().numpy())
    exps = raw[16 * b * b:16 * b * b + 4 * b].view(torch.int32).cpu().numpy()
    return planes, exps


def split_op_graph(S, mats, b):
    """Graph: TRSM(I, M) with prec F64_OZAKI for every matrix M in mats (each
    gets slot i of a fresh store).  Returns graph, store, slot bytes, handles."""
    slot = S.lib.spx_ozaki_slot_bytes(b)
    store = torch.zeros(len(mats) * slot, dtype=torch.uint8, device="cuda")
    g = S.Graph()
    g.register_ozaki(store.data_ptr(), len(mats), b)
    hs = []
    for i, M in enumerate(mats):
        K = M.shape[1]
        eye = torch.eye(K, dtype=torch.float64, device="cuda")
        g._keep.append(eye)
        hI = g.register_tensor(eye)
        hM = g.register(M.data_ptr(), M.shape[0], K, M.stride(0), S.DT_F64,
                        store.data_ptr() + i * slot, b)
        g.insert(S.OP_TRSM, [hI, hM], [S.READ, S.WRITE], prec=S.F64_OZAKI)
        hs.append(hM)
    g._keep.append(store)
    return g, store, slot, hs


def spread_rows(rng, m, K, lo=-30, hi=30):
    A = rng.standard_normal((m, K)) * np.exp2(rng.integers(lo, hi, size=(m, 1)))
    if m > 3:
        A[2] = 0.0
        A[3] *= np.exp2(rng.integers(-45, 0, size=K))
    return A


def worst_case(m, K):
    X = 63 * 128 ** 7 + 64 * sum(128 ** j for j in range(7))
    return np.full((m, K), -X / 2.0 ** 55)


def check_split(store, slot, i, b, M):
    e, D = Z.split(M)
    planes, exps = slot_view(store, slot, i, b)
    m, K = M.shape
    assert np.array_equal(exps[:m], e.astype(np.int32))
    assert np.array_equal(planes[:, :m, :K], D.astype(np.float32))
    assert not planes[:, :m, K:].any()  # the K padding is zero


@pytest.mark.parametrize("m,n,K", [(128, 32, 512), (200, 70, 512), (77, 33, 64), (512, 512, 512),
                                   (256, 96, 40), (33, 130, 200)])
def test_gemm_op_bit_exact(S, m, n, K):
    rng = np.random.default_rng(m * 1000 + n + K)
    A = spread_rows(rng, m, K)
    B = spread_rows(rng, n, K)
    C = rng.standard_normal((m, n))
    b = r32(max(m, n, K))
    Ad, Bd, Cd = (torch.from_numpy(x.copy()).cuda() for x in (A, B, C))
    g, store, slot, (hA, hB) = split_op_graph(S, [Ad, Bd], b)
    hC = g.register_tensor(Cd)
    g.insert(S.OP_GEMM_NT_SUB, [hA, hB, hC], [S.READ, S.READ, S.WRITE], prec=S.F64_OZAKI)
    assert g.run()[0] == 0
    torch.cuda.synchronize()
    assert np.array_equal(Ad.cpu().numpy(), A) and np.array_equal(Bd.cpu().numpy(), B)
    check_split(store, slot, 0, b, A)
    check_split(store, slot, 1, b, B)
    assert np.array_equal(Cd.cpu().numpy(), Z.gemm_nt_sub(C, A, B))
    g.close()


@pytest.mark.parametrize("m,K", [(512, 512), (300, 96), (40, 512)])
def test_syrk_op_bit_exact(S, m, K):
    rng = np.random.default_rng(m + K)
    L = spread_rows(rng, m, K, -8, 8)
    C = rng.standard_normal((m, m))
    b = r32(max(m, K))
    Ld, Cd = (torch.from_numpy(x.copy()).cuda() for x in (L, C))
    g, store, slot, (hL,) = split_op_graph(S, [Ld], b)
    hC = g.register_tensor(Cd)
    g.insert(S.OP_SYRK, [hL, hC], [S.READ, S.WRITE], prec=S.F64_OZAKI)
    assert g.run()[0] == 0
    torch.cuda.synchronize()
    check_split(store, slot, 0, b, L)
    assert np.array_equal(Cd.cpu().numpy(), Z.syrk_lower(C, L))
    g.close()


def test_worst_case_accumulation_exact(S):
    """Every digit -64 (the top one -63), K = 512: the digit sums reach
    P_7 = 16 711 680, within 2^16 of 2^24; the tensor cores must add them
    exactly for the result to match."""
    A = worst_case(128, 512)
    B = worst_case(64, 512)
    B[5::7] *= -1.0
    C = np.zeros((128, 64))
    b = 512
    Ad, Bd, Cd = (torch.from_numpy(x.copy()).cuda() for x in (A, B, C))
    g, store, slot, (hA, hB) = split_op_graph(S, [Ad, Bd], b)
    hC = g.register_tensor(Cd)
    g.insert(S.OP_GEMM_NT_SUB, [hA, hB, hC], [S.READ, S.READ, S.WRITE], prec=S.F64_OZAKI)
    assert g.run()[0] == 0
    torch.cuda.synchronize()
    want = Z.gemm_nt_sub(C, A, B)
    assert np.array_equal(Cd.cpu().numpy(), want)
    g.close()


def run_ozaki(S, A_np, b, X_np=None, lookahead=True, **cfg):
    from paper_2308_15964_b300 import cholesky
    A = torch.from_numpy(np.ascontiguousarray(A_np)).cuda()
    X = torch.from_numpy(np.ascontiguousarray(X_np)).cuda() if X_np is not None else None
    g = S.Graph(**cfg)
    cholesky.cholesky_ozaki_graph(g, A, b, X, lookahead=lookahead)
    rc, info = g.run()
    torch.cuda.synchronize()
    return rc, info, A.cpu().numpy(), (X.cpu().numpy() if X is not None else None), g


def rel_entry_err(L, Lref):
    L, Lref = np.tril(L), np.tril(Lref)
    return np.abs(L - Lref).max() / np.abs(Lref).max()


@pytest.mark.parametrize("n,b,nrhs", [(512, 64, 1), (1000, 128, 2), (33, 32, 1), (700, 96, 3),
                                      (2048, 512, 1), (1024, 256, 2)])
def test_factor_solve_vs_oracle(S, n, b, nrhs):
    A = inputs.spd_matrix(n, 1.0, seed=1).numpy()
    B = inputs.rhs(n, nrhs, seed=1).numpy()
    rc, info, L, X, g = run_ozaki(S, A, b, B)
    assert rc == 0 and info == 0
    Lo, Xo = A.copy(), B.copy()
    assert O.tiled_cholesky(Lo, b, Xo) == 0
    assert rel_entry_err(L, Lo) <= 1e-12
    assert O.solve_backward_error(A, X, B).max() <= 1e-14
    if n <= 1024:
        assert O.factor_backward_error(A, L) <= 1e-14
    assert np.array_equal(np.triu(L, 1), np.triu(A, 1))
    g.close()


@pytest.mark.parametrize("n,b", [(192, 64), (200, 64), (130, 32)])
def test_integer_factor_bit_exact(S, n, b):
    rng = np.random.default_rng(n)
    L0 = np.tril(rng.integers(-1, 2, size=(n, n)).astype(np.float64), -1) + np.eye(n)
    A = L0 @ L0.T
    x0 = rng.integers(-3, 4, size=(n, 2)).astype(np.float64)
    rc, info, L, X, g = run_ozaki(S, A, b, A @ x0)
    assert rc == 0
    assert np.array_equal(np.tril(L), L0)
    assert np.array_equal(X, x0)
    g.close()


def test_diagonal_bit_exact(S):
    n = 320
    e = (np.arange(n) % 9) - 4
    rc, info, L, _, g = run_ozaki(S, np.diag(4.0 ** e), 64)
    assert rc == 0 and info == 0
    assert np.array_equal(np.tril(L), np.diag(2.0 ** e))
    g.close()


@pytest.mark.parametrize("col", [0, 100, 255])
def test_not_spd_info(S, col):
    n = 256
    A = inputs.spd_matrix(n, 1.0, seed=3).numpy()
    A[col, col] = -1.0
    Lo = A.copy()
    info_o = O.tiled_cholesky(Lo, 64)
    rc, info, _, _, g = run_ozaki(S, A, 64)
    assert info == info_o and info > 0
    g.close()


def test_determinism_and_executors(S):
    n, b = 1536, 256
    A = inputs.spd_matrix(n, 0.1, seed=2).numpy()
    B = inputs.rhs(n, 2, seed=2).numpy()
    outs = []
    for cfg in ({}, {}, {"executor": S.EXEC_PER_TASK}, {"executor": S.EXEC_STREAMS},
                {"num_ctas": 37}):
        rc, info, L, X, g = run_ozaki(S, A, b, B, **cfg)
        assert rc == 0 and info == 0
        outs.append((L, X))
        g.close()
    for L, X in outs[1:]:
        assert np.array_equal(L, outs[0][0]) and np.array_equal(X, outs[0][1])


@pytest.mark.slow
def test_scale_16384_sampled(S):
    """The benchmark's configuration (n = 16384, tile 512, split trailing
    updates): the oracle's Freivalds probe of the factor and the oracle's
    backward error of the solve, as for the FP64 path."""
    from paper_2308_15964_b300 import cholesky
    n, b = 16384, 512
    A = inputs.spd_matrix(n, 0.1, seed=2, device="cuda")
    A_host = A.cpu().numpy()
    B = inputs.rhs(n, 1, seed=2, device="cuda")
    B_host = B.cpu().numpy()
    g = S.Graph()
    cholesky.cholesky_ozaki_graph(g, A, b, B)
    rc, info = g.run()
    assert rc == 0 and info == 0
    L = A.cpu().numpy()
    X = B.cpu().numpy()
    for s in range(2):
        assert O.freivalds(A_host, L, inputs.gaussian(n, 100 + s)) <= 1e-14
    assert O.solve_backward_error(A_host, X, B_host).max() <= 1e-14
    g.close()


@pytest.mark.parametrize("n,b", [(1000, 128), (2048, 512)])
def test_bottom_level_priorities_bit_identical(S, n, b):
    """Critical-path priorities change the order and part sizes only: the
    split path's factor and solve are bit-identical to the look-ahead
    marks'."""
    A = inputs.spd_matrix(n, 1.0, seed=n).numpy()
    X = inputs.rhs(n, 2, seed=n).numpy()
    rc1, _, L1, X1, g1 = run_ozaki(S, A, b, X)
    rc2, _, L2, X2, g2 = run_ozaki(S, A, b, X, priorities=1)
    assert rc1 == rc2 == 0
    assert np.array_equal(L1, L2) and np.array_equal(X1, X2)
    g1.close()
    g2.close()


# --- inverse panels: TRTRI (FP64) + split, TRSM_INV as a split product --------

@pytest.mark.parametrize("m,bk", [(512, 512), (200, 96), (77, 64)])
def test_trsm_inv_op_bit_exact(S, m, bk):
    """TRTRI with the split prec inverts L (FP64) and splits V; TRSM_INV with
    the split prec splits A, stores A V^T by the split product and splits
    the result.  V against the oracle's TRTRI (FP64 rounding), every digit
    plane, exponent and product bit for bit against the oracle."""
    Lkk = inputs.spd_matrix(bk, 1.0, seed=m + bk).numpy()
    assert O.potrf(Lkk) == 0
    Lkk = np.tril(Lkk)
    A = np.random.default_rng(m).standard_normal((m, bk))
    b = r32(max(m, bk))
    slot = S.lib.spx_ozaki_slot_bytes(b)
    store = torch.zeros(2 * slot, dtype=torch.uint8, device="cuda")
    Ld = torch.from_numpy(Lkk.copy()).cuda()
    Vd = torch.zeros((bk, bk), dtype=torch.float64, device="cuda")
    Ad = torch.from_numpy(A.copy()).cuda()
    g = S.Graph()
    g.register_ozaki(store.data_ptr(), 2, b)
    hL = g.register_tensor(Ld)
    hV = g.register(Vd.data_ptr(), bk, bk, bk, S.DT_F64, store.data_ptr() + slot, b)
    hA = g.register(Ad.data_ptr(), m, bk, bk, S.DT_F64, store.data_ptr(), b)
    g.insert(S.OP_TRTRI, [hL, hV], [S.READ, S.WRITE], prec=S.F64_OZAKI)
    g.insert(S.OP_TRSM_INV, [hV, hA], [S.READ, S.WRITE], prec=S.F64_OZAKI)
    assert g.run()[0] == 0
    torch.cuda.synchronize()
    V = Vd.cpu().numpy()
    Vo = O.trtri(Lkk)
    assert np.abs(V - Vo).max() <= 1e-12 * np.abs(Vo).max()
    check_split(store, slot, 1, b, V)
    X = Ad.cpu().numpy()
    assert np.array_equal(X, Z.products(A, V))
    check_split(store, slot, 0, b, X)
    g.close()


def bidiag_lower(n, b, seed):
    """Unit lower L0 with diagonal tiles I - S (inverses: lower triangles of
    ones) and off-diagonal entries in {-1, 0, 1}: every inverse, product and
    partial sum is a small integer."""
    rng = np.random.default_rng(seed)
    L = np.tril(rng.integers(-1, 2, size=(n, n)).astype(np.float64), -1)
    for k in range(0, n, b):
        e = min(n, k + b)
        L[k:e, k:e] = np.eye(e - k) - np.eye(e - k, k=-1)
    return L


def run_ozaki_inv(S, A_np, b, X_np=None, **cfg):
    from paper_2308_15964_b300 import cholesky
    n = A_np.shape[0]
    A = torch.from_numpy(np.ascontiguousarray(A_np)).cuda()
    X = torch.from_numpy(np.ascontiguousarray(X_np)).cuda() if X_np is not None else None
    V = torch.zeros((n, b), dtype=torch.float64, device="cuda")
    g = S.Graph(**cfg)
    cholesky.cholesky_ozaki_graph(g, A, b, X, V=V)
    rc, info = g.run()
    torch.cuda.synchronize()
    return rc, info, A.cpu().numpy(), (X.cpu().numpy() if X is not None else None), V, g


@pytest.mark.parametrize("n,b", [(1024, 256), (1000, 256), (640, 128)])
def test_inverse_panels_integer_bit_exact(S, n, b):
    L0 = bidiag_lower(n, b, n + b)
    A = L0 @ L0.T
    x0 = np.random.default_rng(3).integers(-3, 4, size=(n, 2)).astype(np.float64)
    outs = []
    for ex in (S.EXEC_PERSISTENT, S.EXEC_PER_TASK):
        rc, info, L, X, V, g = run_ozaki_inv(S, A, b, A @ x0, executor=ex)
        assert rc == 0 and info == 0
        assert np.array_equal(np.tril(L), L0)
        assert np.array_equal(X, x0)
        Vh = V.cpu().numpy()
        for k in range(0, n, b):
            bk = min(b, n - k)
            assert np.array_equal(Vh[k:k + bk, :bk], np.tril(np.ones((bk, bk))))
        outs.append(L)
        g.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("n,b,nrhs", [(512, 64, 1), (1000, 128, 2), (700, 96, 3), (2048, 512, 1),
                                      (4096, 512, 2)])
def test_inverse_panels_vs_oracle(S, n, b, nrhs):
    A = inputs.spd_matrix(n, 0.1, seed=5).numpy()
    B = inputs.rhs(n, nrhs, seed=5).numpy()
    rc, info, L, X, V, g = run_ozaki_inv(S, A, b, B)
    assert rc == 0 and info == 0
    Lo = A.copy()
    assert O.tiled_cholesky(Lo, b) == 0
    assert rel_entry_err(L, Lo) <= 1e-12
    assert O.solve_backward_error(A, X, B).max() <= 1e-14
    if n <= 2048:
        assert O.factor_backward_error(A, L) <= 1e-14
    g.close()


@pytest.mark.slow
def test_inverse_panels_16384_sampled(S):
    from paper_2308_15964_b300 import cholesky
    n, b = 16384, 512
    A = inputs.spd_matrix(n, 0.1, seed=2, device="cuda")
    A_host = A.cpu().numpy()
    B = inputs.rhs(n, 1, seed=2, device="cuda")
    B_host = B.cpu().numpy()
    V = torch.zeros((n, b), dtype=torch.float64, device="cuda")
    g = S.Graph()
    cholesky.cholesky_ozaki_graph(g, A, b, B, V=V)
    rc, info = g.run()
    assert rc == 0 and info == 0
    L = A.cpu().numpy()
    X = B.cpu().numpy()
    for s in range(2):
        assert O.freivalds(A_host, L, inputs.gaussian(n, 100 + s)) <= 1e-14
    assert O.solve_backward_error(A_host, X, B_host).max() <= 1e-14
    g.close()


# --- the critical panel tile solved inside POTRF (POTRF_PANEL) -----------------

@pytest.mark.parametrize("n,m,b", [(512, 512, 512), (256, 100, 256), (320, 320, 320)])
def test_potrf_panel_op(S, n, m, b):
    """POTRF_PANEL (FP64) against the oracle's POTRF then TRSM (its
    definition), and bit-identical to the POTRF and TRSM tasks on the GPU."""
    Afull = inputs.spd_matrix(n + m, 1.0, seed=n + m).numpy()
    P0 = np.ascontiguousarray(Afull[:n, :n])
    Q0 = np.ascontiguousarray(Afull[n:, :n])
    outs = []
    for fused in (True, False):
        Pd = torch.from_numpy(P0.copy()).cuda()
        Qd = torch.from_numpy(Q0.copy()).cuda()
        g = S.Graph()
        hp, hq = g.register_tensor(Pd), g.register_tensor(Qd)
        if fused:
            g.insert(S.OP_POTRF_PANEL, [hp, hq], [S.WRITE, S.WRITE], 2)
        else:
            g.insert(S.OP_POTRF, [hp], [S.WRITE], 2)
            g.insert(S.OP_TRSM, [hp, hq], [S.READ, S.WRITE], 2)
        assert g.run()[0] == 0
        torch.cuda.synchronize()
        outs.append((Pd.cpu().numpy(), Qd.cpu().numpy()))
        g.close()
    assert np.array_equal(np.tril(outs[0][0]), np.tril(outs[1][0]))
    assert np.array_equal(outs[0][1], outs[1][1])
    # the oracle: tiles (0, 0) and (1, 0) of the (n + m) square matrix, tile n
    mats = {"A": Afull.copy()}
    info = O.execute([(O.POTRF_PANEL, [(("A", 0, 0), O.WRITE), (("A", 1, 0), O.WRITE)], 0)], mats,
                     n)
    assert info == 0
    Lo = np.tril(mats["A"][:n, :n])
    Qo = mats["A"][n:, :n]
    assert np.abs(np.tril(outs[0][0]) - Lo).max() <= 1e-12 * np.abs(Lo).max()
    assert np.abs(outs[0][1] - Qo).max() <= 1e-12 * np.abs(Qo).max()


@pytest.mark.parametrize("n,b,inverse", [(2048, 512, True), (1000, 128, True), (1536, 256, False)])
def test_fused_panel_bit_identical(S, n, b, inverse):
    """The split Cholesky with the fused critical panel equals the unfused one
    bit for bit, and the oracle within the FP64 tolerances."""
    from paper_2308_15964_b300 import cholesky
    A = inputs.spd_matrix(n, 0.1, seed=9).numpy()
    B = inputs.rhs(n, 2, seed=9).numpy()
    res = []
    for fuse in (True, False):
        Ad = torch.from_numpy(A.copy()).cuda()
        Xd = torch.from_numpy(B.copy()).cuda()
        V = torch.zeros((n, b), dtype=torch.float64, device="cuda") if inverse else None
        g = S.Graph()
        cholesky.cholesky_ozaki_graph(g, Ad, b, Xd, V=V, fuse_panel=fuse)
        rc, info = g.run()
        assert rc == 0 and info == 0
        torch.cuda.synchronize()
        res.append((Ad.cpu().numpy(), Xd.cpu().numpy()))
        g.close()
    assert np.array_equal(np.tril(res[0][0]), np.tril(res[1][0]))
    assert np.array_equal(res[0][1], res[1][1])
    Lo = A.copy()
    assert O.tiled_cholesky(Lo, b) == 0
    assert rel_entry_err(res[0][0], Lo) <= 1e-12
    assert O.solve_backward_error(A, res[0][1], B).max() <= 1e-14


def test_fused_panel_integer_and_not_spd(S):
    from paper_2308_15964_b300 import cholesky
    n, b = 1024, 256
    L0 = bidiag_lower(n, b, 77)
    A = L0 @ L0.T
    Ad = torch.from_numpy(A.copy()).cuda()
    V = torch.zeros((n, b), dtype=torch.float64, device="cuda")
    g = S.Graph()
    cholesky.cholesky_ozaki_graph(g, Ad, b, V=V, fuse_panel=True)
    assert g.run()[0] == 0
    torch.cuda.synchronize()
    assert np.array_equal(np.tril(Ad.cpu().numpy()), L0)
    g.close()
    A2 = inputs.spd_matrix(512, 1.0, seed=3).numpy()
    A2[300, 300] = -1.0
    Lo = A2.copy()
    info_o = O.tiled_cholesky(Lo, 128)
    Ad = torch.from_numpy(A2.copy()).cuda()
    g = S.Graph()
    cholesky.cholesky_ozaki_graph(g, Ad, 128, V=torch.zeros((512, 128), dtype=torch.float64,
                                                            device="cuda"), fuse_panel=True)
    rc, info = g.run()
    assert info == info_o and info > 0
    g.close()


# --- the NN form: SPLIT / SPLIT_T tasks and GEMM_NN_ADD on split products ----

def split_nn_graph(S, Ad, Bd, b):
    """Graph: SPLIT(A) into slot 0, SPLIT_T(B) into slot 1 of a fresh store."""
    slot = S.lib.spx_ozaki_slot_bytes(b)
    store = torch.full((2 * slot,), 0x7F, dtype=torch.uint8, device="cuda")  # not zeros
    g = S.Graph()
    g.register_ozaki(store.data_ptr(), 2, b)
    hA = g.register(Ad.data_ptr(), Ad.shape[0], Ad.shape[1], Ad.stride(0), S.DT_F64,
                    store.data_ptr(), b)
    hB = g.register(Bd.data_ptr(), Bd.shape[0], Bd.shape[1], Bd.stride(0), S.DT_F64,
                    store.data_ptr() + slot, b)
    g.insert(S.OP_SPLIT, [hA], [S.WRITE], prec=S.F64_OZAKI)
    g.insert(S.OP_SPLIT_T, [hB], [S.WRITE], prec=S.F64_OZAKI)
    g._keep.append(store)
    return g, store, slot, hA, hB


@pytest.mark.parametrize("m,n,K", [(128, 64, 512), (200, 70, 136), (33, 130, 200),
                                   (512, 512, 512), (77, 33, 40)])
def test_gemm_nn_op_bit_exact(S, m, n, K):
    """SPLIT writes the oracle's row split of A, SPLIT_T the split of B^T
    (column exponents, K = B's rows, zero K padding over a store that starts
    non-zero); GEMM_NN_ADD then equals the oracle's C + A B bit for bit."""
    rng = np.random.default_rng(7 * m + 3 * n + K)
    A = spread_rows(rng, m, K)
    B = np.ascontiguousarray(spread_rows(rng, n, K).T)  # columns of spread magnitudes
    C = rng.standard_normal((m, n))
    b = r32(max(m, n, K))
    Ad, Bd, Cd = (torch.from_numpy(x.copy()).cuda() for x in (A, B, C))
    g, store, slot, hA, hB = split_nn_graph(S, Ad, Bd, b)
    hC = g.register_tensor(Cd)
    g.insert(S.OP_GEMM_NN_ADD, [hA, hB, hC], [S.READ, S.READ, S.WRITE], prec=S.F64_OZAKI)
    assert g.run()[0] == 0
    torch.cuda.synchronize()
    assert np.array_equal(Ad.cpu().numpy(), A) and np.array_equal(Bd.cpu().numpy(), B)
    check_split(store, slot, 0, b, A)
    check_split(store, slot, 1, b, B.T)
    assert np.array_equal(Cd.cpu().numpy(), Z.gemm_nn_add(C, A, B))
    g.close()


def test_gemm_nn_worst_case_exact(S):
    """The worst digit sums (P_7 just below 2^24) through the NN form."""
    A = worst_case(128, 512)
    B = np.ascontiguousarray(worst_case(64, 512).T)
    B[:, 3::5] *= -1.0
    C = np.zeros((128, 64))
    Ad, Bd, Cd = (torch.from_numpy(x.copy()).cuda() for x in (A, B, C))
    g, store, slot, hA, hB = split_nn_graph(S, Ad, Bd, 512)
    hC = g.register_tensor(Cd)
    g.insert(S.OP_GEMM_NN_ADD, [hA, hB, hC], [S.READ, S.READ, S.WRITE], prec=S.F64_OZAKI)
    assert g.run()[0] == 0
    torch.cuda.synchronize()
    assert np.array_equal(Cd.cpu().numpy(), Z.gemm_nn_add(C, A, B))
    g.close()


def test_gemm_nn_rejects_bad_use(S):
    """SPLIT needs the split prec and a slot; the split GEMM is not atomic."""
    Ad = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    Bd, Cd = torch.zeros_like(Ad), torch.zeros_like(Ad)
    g, store, slot, hA, hB = split_nn_graph(S, Ad, Bd, 64)
    hC = g.register_tensor(Cd)
    with pytest.raises(S.SpxError):
        g.insert(S.OP_SPLIT, [hA], [S.WRITE], prec=S.F64)
    with pytest.raises(S.SpxError):
        g.insert(S.OP_SPLIT, [hC], [S.WRITE], prec=S.F64_OZAKI)  # no slot
    with pytest.raises(S.SpxError):
        g.insert(S.OP_GEMM_NN_ADD, [hA, hB, hC], [S.READ, S.READ, S.ATOMIC_WRITE],
                 prec=S.F64_OZAKI)
    with pytest.raises(S.SpxError):
        g.insert(S.OP_GEMM_NN_ADD, [hA, hC, hB], [S.READ, S.READ, S.WRITE], prec=S.F64_OZAKI)
    g.close()


def run_gemm_ozaki(S, A, B, C, b, commutative=False, **cfg):
    from paper_2308_15964_b300 import cholesky
    Ad, Bd, Cd = (torch.from_numpy(x.copy()).cuda() for x in (A, B, C))
    g = S.Graph(**cfg)
    nt = cholesky.gemm_ozaki_graph(g, Ad, Bd, Cd, b, commutative=commutative)
    rc = g.run()[0]
    torch.cuda.synchronize()
    out = Cd.cpu().numpy()
    g.close()
    return rc, nt, out


@pytest.mark.parametrize("n,b", [(600, 128), (512, 256), (96, 32)])
def test_gemm_dag_vs_oracle(S, n, b):
    """spx_gemm_insert_ozaki (WRITE on C_ij: k in order) bit for bit against
    the oracle's tiled split GEMM, with the persistent and per-task
    executors; ragged last tiles."""
    rng = np.random.default_rng(n + b)
    A = inputs.uniform((n, n), seed=n).numpy()
    B = rng.uniform(-1, 1, (n, n)) * np.exp2(rng.integers(-20, 20, size=(1, n)))
    C = rng.uniform(-1, 1, (n, n))
    want = Z.tiled_gemm_nn_add(A, B, C.copy(), b)
    T = -(-n // b)
    for ex in (S.EXEC_PERSISTENT, S.EXEC_PER_TASK):
        rc, nt, got = run_gemm_ozaki(S, A, B, C, b, executor=ex)
        assert rc == 0 and nt == 2 * T * T + T ** 3
        assert np.array_equal(got, want), ex
    # FP64's accuracy against the exact-enough reference
    ref = C + A @ B
    scale = np.abs(A) @ np.abs(B) + np.abs(C)
    assert np.max(np.abs(want - ref) / scale) < 1e-14


def test_gemm_dag_commutative(S):
    """COMMUTATIVE_WRITE: the k order of a block is free, so the result
    equals the oracle's to rounding, and bit for bit on integer inputs
    (every split product and sum then exact)."""
    n, b = 512, 128
    rng = np.random.default_rng(5)
    A = rng.uniform(-1, 1, (n, n))
    B = rng.uniform(-1, 1, (n, n))
    C = rng.uniform(-1, 1, (n, n))
    rc, _, got = run_gemm_ozaki(S, A, B, C, b, commutative=True)
    assert rc == 0
    want = Z.tiled_gemm_nn_add(A, B, C.copy(), b)
    assert np.max(np.abs(got - want)) <= 4 * 2.0 ** -52 * np.max(np.abs(want))
    Ai = rng.integers(-2 ** 19, 2 ** 19, size=(n, n)).astype(np.float64)
    Bi = rng.integers(-2 ** 19, 2 ** 19, size=(n, n)).astype(np.float64)
    Ci = rng.integers(-2 ** 30, 2 ** 30, size=(n, n)).astype(np.float64)
    rc, _, got = run_gemm_ozaki(S, Ai, Bi, Ci, b, commutative=True)
    assert rc == 0
    exact = (Ci.astype(np.int64) + Ai.astype(np.int64) @ Bi.astype(np.int64)).astype(np.float64)
    assert np.array_equal(got, exact)


def test_gemm_dag_8192_sampled(S):
    """The benchmark's size (n = 8192, tile 512, entries uniform[-1, 1]),
    WRITE form: sampled entries against the oracle's split products taken
    one entry and one k at a time, in the tasks' order."""
    from paper_2308_15964_b300 import cholesky
    n, b = 8192, 512
    Ad, Bd, Cd = (inputs.uniform((n, n), sd, device="cuda") for sd in (3, 4, 5))
    A, B, C = Ad.cpu(), Bd.cpu(), Cd.cpu()
    g = S.Graph()
    cholesky.gemm_ozaki_graph(g, Ad, Bd, Cd, b)
    assert g.run()[0] == 0
    torch.cuda.synchronize()
    got = Cd.cpu().numpy()
    g.close()
    An, Bn, Cn = A.numpy(), B.numpy(), C.numpy()
    rng = np.random.default_rng(1)
    rows = np.concatenate([[0, n - 1, 511, 512], rng.integers(0, n, 12)])
    cols = np.concatenate([[n - 1, 0, 512, 511], rng.integers(0, n, 12)])
    for r, c in zip(rows, cols):
        v = Cn[r, c]
        for k in range(n // b):
            ks = slice(k * b, (k + 1) * b)
            v = v + Z.products(An[r:r + 1, ks], Bn[ks, c][None, :])[0, 0]
        assert got[r, c] == v, (r, c)
