"""GPU parity of the FP64 tiled Cholesky + solve against the oracle.

Tolerances (stated for the FP64 path): max relative entry error of L
<= 1e-12 against the oracle's L; normwise backward error of every solve
<= 1e-14; factor backward error <= 1e-14.  Exact pins: power-of-4 diagonal
and integer unit-lower factors are reproduced bit for bit.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2308_15964_b300 import inputs
from tests._gpu import need_cuda, run_cholesky, spx_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    need_cuda()
    return spx_mod()


def rel_entry_err(L, Lref):
    L, Lref = np.tril(L), np.tril(Lref)
    return np.abs(L - Lref).max() / np.abs(Lref).max()


@pytest.mark.parametrize("n,b,nrhs", [(512, 64, 1), (100, 32, 3), (1000, 128, 2), (64, 64, 1), (1024, 256, 2),
                                      (33, 8, 1), (700, 256, 5), (2048, 512, 1)])
def test_factor_solve_vs_oracle(S, n, b, nrhs):
    A = inputs.spd_matrix(n, 1.0, seed=1).numpy()
    B = inputs.rhs(n, nrhs, seed=1).numpy()
    rc, info, L, X, g = run_cholesky(A, b, B)
    assert rc == 0 and info == 0
    Lo, Xo = A.copy(), B.copy()
    assert O.tiled_cholesky(Lo, b, Xo) == 0
    assert rel_entry_err(L, Lo) <= 1e-12
    assert O.solve_backward_error(A, X, B).max() <= 1e-14
    if n <= 1024:
        assert O.factor_backward_error(A, L) <= 1e-14
    # strict upper triangle of the diagonal tiles and upper tiles untouched
    assert np.array_equal(np.triu(L, 1), np.triu(A, 1))
    g.close()


@pytest.mark.parametrize("n,b", [(192, 64), (200, 64), (130, 32)])
def test_integer_factor_bit_exact(S, n, b):
    rng = np.random.default_rng(n)
    L0 = np.tril(rng.integers(-1, 2, size=(n, n)).astype(np.float64), -1) + np.eye(n)
    A = L0 @ L0.T
    x0 = rng.integers(-3, 4, size=(n, 2)).astype(np.float64)
    rc, info, L, X, g = run_cholesky(A, b, A @ x0)
    assert rc == 0
    assert np.array_equal(np.tril(L), L0)
    assert np.array_equal(X, x0)
    g.close()


def test_diagonal_bit_exact(S):
    n, b = 300, 64
    e = (np.arange(n) % 11) - 5
    A = np.diag(4.0 ** e)
    rc, info, L, _, g = run_cholesky(A, b)
    assert rc == 0 and np.array_equal(np.tril(L), np.diag(2.0 ** e))
    g.close()


@pytest.mark.parametrize("col", [1, 64, 65, 150, 200])
def test_not_spd_info(S, col):
    n, b = 200, 64
    A = inputs.spd_matrix(n, 1.0, seed=2).numpy()
    A[col - 1, col - 1] = -1.0
    expect = O.tiled_cholesky(A.copy(), b)
    assert expect == O.potrf(A.copy())
    rc, info, _, _, g = run_cholesky(A, b)
    assert rc == S.NOT_SPD and info == expect
    g.close()
    for ex in (S.EXEC_PER_TASK, S.EXEC_STREAMS):
        rc, info, _, _, g = run_cholesky(A, b, executor=ex)
        assert rc == S.NOT_SPD and info == expect
        g.close()


def test_determinism_and_executors(S):
    n, b = 768, 128
    A = inputs.spd_matrix(n, 1.0, seed=4).numpy()
    B = inputs.rhs(n, 3, seed=4).numpy()
    ref = run_cholesky(A, b, B)
    outs = [run_cholesky(A, b, B), run_cholesky(A, b, B, executor=S.EXEC_PER_TASK),
            run_cholesky(A, b, B, executor=S.EXEC_STREAMS),
            run_cholesky(A, b, B, no_split=True), run_cholesky(A, b, B, num_ctas=3),
            run_cholesky(A, b, B, lookahead=False), run_cholesky(A, b, B, lookahead=2)]
    for o in outs:
        assert o[0] == 0
        assert np.array_equal(o[2], ref[2]) and np.array_equal(o[3], ref[3])
        o[4].close()
    ref[4].close()


@pytest.mark.parametrize("mode", ["write", "commutative", "atomic"])
def test_gemm_dag_vs_oracle(S, mode):
    """The tiled GEMM DAG with a WRITE chain, a COMMUTATIVE_WRITE run or an
    ATOMIC_WRITE run on each C block (atomic: all tasks of a block run at
    once and add with atomic FP64 additions) against the oracle."""
    from paper_2308_15964_b300 import cholesky
    n, b = 320, 64
    A = inputs.uniform((n, n), 3).numpy()
    B = inputs.uniform((n, n), 4).numpy()
    C = inputs.uniform((n, n), 5).numpy()
    Co = C.copy()
    O.tiled_gemm(A, B, Co, b)
    dA, dB, dC = (torch.from_numpy(x).cuda() for x in (A, B, C))
    g = S.Graph()
    cholesky.gemm_graph(g, dA, dB, dC, b, commutative=mode == "commutative",
                        atomic=mode == "atomic")
    if mode == "atomic":
        g.derive()
        assert g.sizes()[1] == 0        # no edges: every block is one atomic run
    rc, _ = g.run()
    assert rc == 0
    got = dC.cpu().numpy()
    bound = 2 * n * 2.2e-16 * (np.abs(A) @ np.abs(B) + np.abs(C))
    assert (np.abs(got - Co) <= bound).all()
    g.close()


def test_spin_watchdog_timeout(S):
    # a task that spins longer than the watchdog: the device gives up, sets
    # SPX_ERR_TIMEOUT and the kernel returns (no hang, context usable after)
    g = S.Graph(watchdog_ns=200_000_000)
    h = g.register(0x7f0000000000, 8, 8, 8)
    t0 = g.insert(S.OP_SPIN, [h], [S.WRITE])
    g.set_arg(t0, 5_000_000_000)
    g.insert(S.OP_NOP, [h], [S.READ])
    rc, _ = g.run()
    assert rc == S.ERR_TIMEOUT
    g.close()
    # and a short spin completes
    g = S.Graph(watchdog_ns=2_000_000_000)
    h = g.register(0x7f0000000000, 8, 8, 8)
    t0 = g.insert(S.OP_SPIN, [h], [S.WRITE])
    g.set_arg(t0, 1_000_000)
    rc, _ = g.run()
    assert rc == 0
    g.close()


def test_queue_full(S):
    g = S.Graph(queue_capacity=2)
    hs = [g.register(0x7f0000000000 + 4096 * i, 8, 8, 8) for i in range(8)]
    w = g.insert(S.OP_NOP, hs, [S.WRITE] * 8)
    for h in hs:
        g.insert(S.OP_NOP, [h], [S.READ])           # 8 successors released together
    rc, _ = g.run()
    assert rc == S.ERR_QUEUE_FULL
    g.close()
    del w


def test_trace(S):
    n, b = 256, 64
    A = inputs.spd_matrix(n, 1.0, seed=5).numpy()
    rc, info, L, _, g = run_cholesky(A, b, trace=True)
    assert rc == 0
    tr = g.trace()
    rp, col, _ = g.edges()
    assert (tr[:, 1] >= tr[:, 0]).all() and (tr[:, 3] >= 1).all()
    for u in range(len(rp) - 1):
        for p in range(rp[u], rp[u + 1]):
            assert tr[u, 1] <= tr[col[p], 0] + 1000   # successor starts after (clock skew < 1 us)
    g.close()


@pytest.mark.slow
def test_scale_16384_sampled(S):
    """At the benchmark size the oracle cannot factor the matrix; check the
    GPU factor with a Freivalds probe (oracle, O(n^2)) and the solve's
    backward error, both computed on the host by the oracle."""
    from paper_2308_15964_b300 import cholesky
    n, b = 16384, 512
    A = inputs.spd_matrix(n, 0.1, seed=2, device="cuda")
    A_host = A.cpu().numpy()
    B = inputs.rhs(n, 1, seed=2, device="cuda")
    B_host = B.cpu().numpy()
    g = S.Graph()
    cholesky.cholesky_graph(g, A, b, B)
    rc, info = g.run()
    assert rc == 0
    L = A.cpu().numpy()
    X = B.cpu().numpy()
    for s in range(2):
        assert O.freivalds(A_host, L, inputs.gaussian(n, 100 + s)) <= 1e-14
    assert O.solve_backward_error(A_host, X, B_host).max() <= 1e-14
    g.close()


@pytest.mark.parametrize("n,b", [(512, 64), (1000, 128), (2048, 512)])
def test_bottom_level_priorities_bit_identical(S, n, b):
    """Priorities from the critical path (cfg.priorities = 1) change only the
    order of execution and the part sizes, never a tile's arithmetic: factor
    and solve bit-identical to the look-ahead marks, and the ticket order
    respects every edge."""
    A = inputs.spd_matrix(n, 1.0, seed=n)
    X = inputs.rhs(n, 2, seed=n)
    rc1, _, L1, X1, g1 = run_cholesky(A.numpy(), b, X.numpy())
    rc2, _, L2, X2, g2 = run_cholesky(A.numpy(), b, X.numpy(), priorities=1)
    assert rc1 == rc2 == 0
    assert np.array_equal(L1, L2) and np.array_equal(X1, X2)
    ops, prio = g2.task_ops()
    assert (prio == 2).any() and (prio == 0).any()
    rp, col, _ = g2.edges()
    s, e = g2.tickets()
    for u in range(len(rp) - 1):
        for p in range(rp[u], rp[u + 1]):
            assert e[u] < s[col[p]]
    g1.close()
    g2.close()
