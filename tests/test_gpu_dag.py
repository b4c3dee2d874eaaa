"""GPU parity of the device DAG derivation (bit-exact against the oracle) and
of the scheduler's execution invariants (tickets)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2308_15964_b300 import inputs
from tests._golden import load_dag_fixture
from tests._gpu import need_cuda, nop_graph, spx_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    need_cuda()
    return spx_mod()


def check_same(g, ntasks, t, k, m):
    g.derive()
    rp, col, deg = g.edges()
    orp, ocol, odeg = O.derive(ntasks, t, k, m)
    assert np.array_equal(rp, orp)
    assert np.array_equal(col, ocol)
    assert np.array_equal(deg, odeg)
    return rp, col, deg


def check_tickets(g, rp, col, acc=None):
    rc, info = g.run()
    assert rc == 0, rc
    s, e = g.tickets()
    n = len(rp) - 1
    assert (s != 0xFFFFFFFF).all() and (e > s).all()
    for u in range(n):
        for p in range(rp[u], rp[u + 1]):
            assert e[u] < s[col[p]]
    st = g.stats()
    assert st["parts"] >= n
    return s, e


def test_golden_fixture_atomic_maybe(S):
    n, t, k, m, edges, indeg = load_dag_fixture("dag_modes_atomic_maybe.txt")
    g = nop_graph(S, n, t, k, m)
    rp, col, deg = check_same(g, n, t, k, m)
    got = [(u, int(col[p])) for u in range(n) for p in range(rp[u], rp[u + 1])]
    assert got == edges and list(deg) == indeg
    check_tickets(g, rp, col)
    g.close()


@pytest.mark.parametrize("seed", range(12))
def test_random_access_lists_five_modes(S, seed):
    ntask = [3, 40, 300, 2000][seed % 4]
    nkeys = [1, 3, 16][seed % 3]
    t, k, m = inputs.random_access_lists(ntask, nkeys, 5, seed=8800 + seed, nmodes=5)
    n = int(t.max()) + 1
    g = nop_graph(S, n, t, k, m)
    rp, col, _ = check_same(g, n, t, k, m)
    check_tickets(g, rp, col)
    g.close()


def test_golden_fixture(S):
    n, t, k, m, edges, indeg = load_dag_fixture()
    g = nop_graph(S, n, t, k, m)
    rp, col, deg = check_same(g, n, t, k, m)
    got = [(u, int(col[p])) for u in range(n) for p in range(rp[u], rp[u + 1])]
    assert got == edges and list(deg) == indeg
    s, e = check_tickets(g, rp, col)
    # members of the commutative run {3, 4} on x, and {9, 10} on y, never overlap
    for a, b in ((3, 4), (9, 10)):
        assert e[a] < s[b] or e[b] < s[a]
    g.close()


@pytest.mark.parametrize("T", [1, 2, 3, 8, 17, 32])
def test_cholesky_dag(S, T):
    from paper_2308_15964_b300 import cholesky
    b = 8
    n = T * b - (3 if T > 2 else 0)         # ragged last tile
    A = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    X = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    g = S.Graph()
    cholesky.cholesky_graph(g, A, b, X)
    tasks = O.cholesky_tasks(T, b, with_solve=True)
    t, k, m, _ = O.access_arrays(tasks)
    assert g.sizes()[0] == len(tasks)
    rp, col, deg = check_same(g, len(tasks), t, k, m)
    g.close()


@pytest.mark.parametrize("commutative", [False, True])
def test_gemm_dag(S, commutative):
    from paper_2308_15964_b300 import cholesky
    T, b = 16, 8
    A, B, C = (torch.zeros((T * b, T * b), dtype=torch.float64, device="cuda") for _ in range(3))
    g = S.Graph()
    cholesky.gemm_graph(g, A, B, C, b, commutative)
    t, k, m, _ = O.access_arrays(O.gemm_tasks(T, commutative))
    check_same(g, T ** 3, t, k, m)
    g.close()


@pytest.mark.parametrize("seed", range(40))
def test_random_access_lists(S, seed):
    ntask = [1, 2, 5, 30, 200, 1500][seed % 6]
    nkeys = [1, 2, 4, 16, 64][seed % 5]
    t, k, m = inputs.random_access_lists(ntask, nkeys, 6, seed=500 + seed)
    n = int(t.max()) + 1
    g = nop_graph(S, n, t, k, m)
    rp, col, _ = check_same(g, n, t, k, m)
    s, e = check_tickets(g, rp, col)
    # commutative runs: members sharing a key run one at a time
    acc = {}
    for ti, ki, mi in zip(t, k, m):
        acc.setdefault(int(ti), {})
        d = acc[int(ti)]
        d[int(ki)] = int(mi) if int(ki) not in d or d[int(ki)] == int(mi) else 1
    by_key = {}
    for ti in range(n):
        for key, md in acc[ti].items():
            by_key.setdefault(key, []).append((ti, md))
    for key, lst in by_key.items():
        run = []
        for ti, md in lst + [(-1, -1)]:
            if md == 2:
                run.append(ti)
                continue
            iv = sorted((s[x], e[x]) for x in run)
            for (a0, a1), (b0, b1) in zip(iv, iv[1:]):
                assert a1 < b0
            run = []
    g.close()


def test_large_random(S):
    t, k, m = inputs.random_access_lists(40000, 3000, 5, seed=77)
    n = int(t.max()) + 1
    g = nop_graph(S, n, t, k, m)
    rp, col, _ = check_same(g, n, t, k, m)
    check_tickets(g, rp, col)
    g.close()


def test_reexecute_and_dot(S, tmp_path):
    t, k, m = inputs.random_access_lists(50, 6, 3, seed=3)
    n = int(t.max()) + 1
    g = nop_graph(S, n, t, k, m)
    rp, col, _ = check_same(g, n, t, k, m)
    for _ in range(3):
        check_tickets(g, rp, col)
        g.reset()
    path = tmp_path / "g.dot"
    g.write_dot(str(path))
    text = path.read_text()
    assert text.count("->") == len(col) and text.startswith("digraph")
    g.close()


def test_priority_and_ctas(S):
    # a single CTA still finishes a wide graph; high priority entries pop first
    t, k, m = inputs.random_access_lists(300, 10, 3, seed=11)
    n = int(t.max()) + 1
    g = nop_graph(S, n, t, k, m, num_ctas=1)
    rp, col, _ = check_same(g, n, t, k, m)
    check_tickets(g, rp, col)
    assert g.stats()["ctas"] == 1
    g.close()


@pytest.mark.parametrize("commutative", [False, True])
@pytest.mark.parametrize("deps,spin_ns", [(1, 0), (3, 2000), (16, 0)])
def test_overhead_pattern(S, commutative, deps, spin_ns):
    """The engine-overhead graph (T chains of N tasks on d objects each): its
    DAG equals the oracle's for the same access lists, every edge is kept at
    run time, and the commutative tasks of a chain never overlap."""
    import ctypes
    T, N = 7, 5
    g = S.Graph()
    nt = ctypes.c_longlong()
    assert S.lib.spx_overhead_insert(g._h, T, N, deps, int(commutative), spin_ns,
                                     ctypes.byref(nt)) == 0
    assert nt.value == T * N
    mode = O.COMMUTATIVE_WRITE if commutative else O.WRITE
    # oracle view: task j*T + c accesses objects c*deps .. c*deps + deps - 1
    t = np.repeat(np.arange(T * N, dtype=np.uint32), deps)
    k = np.array([(u % T) * deps + d for u in range(T * N) for d in range(deps)], np.uint64)
    m = np.full(T * N * deps, mode, np.int32)
    rp, col, _ = check_same(g, T * N, t, k, m)
    if not commutative:
        assert [(u, int(col[p])) for u in range(T * N) for p in range(rp[u], rp[u + 1])] == \
            [(u, u + T) for u in range(T * (N - 1))]
    else:
        assert len(col) == 0
    s, e = check_tickets(g, rp, col)
    if commutative:
        for c in range(T):
            iv = sorted((s[j * T + c], e[j * T + c]) for j in range(N))
            assert all(iv[i][1] < iv[i + 1][0] for i in range(N - 1))
    g.close()


def test_overhead_pattern_rejects_bad_sizes(S):
    import ctypes
    g = S.Graph()
    nt = ctypes.c_longlong()
    for args in ((0, 4, 1), (4, 0, 1), (4, 4, 0), (4, 4, 17)):
        assert S.lib.spx_overhead_insert(g._h, *args, 0, 0, ctypes.byref(nt)) == S.ERR_INVALID_ARG
    g.close()
