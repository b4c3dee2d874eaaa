"""Pins of the oracle's DAG derivation against facts other than itself.

* a hand-derived graph for all three access modes (tests/golden);
* closed-form counts of the tiled Cholesky DAG (tasks, edges, critical path,
  in-degree pattern) and of the tiled GEMM DAG;
* brute force on small random graphs: the transitive closure of the derived
  edges equals the closure of the pairwise conflict relation of the STF
  model, and no edge joins two members of a READ group or of a COMMUTATIVE run.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2308_15964_b300 import inputs
from tests._golden import load_dag_fixture


def csr_edges(row_ptr, col):
    out = []
    for u in range(len(row_ptr) - 1):
        for p in range(row_ptr[u], row_ptr[u + 1]):
            out.append((u, int(col[p])))
    return out


@pytest.mark.parametrize("name", ["dag_modes_small.txt", "dag_modes_atomic_maybe.txt"])
def test_golden_modes_graph(name):
    n, t, k, m, edges, indeg = load_dag_fixture(name)
    row_ptr, col, deg = O.derive(n, t, k, m)
    assert csr_edges(row_ptr, col) == edges
    assert list(deg) == indeg


def longest_path(n, row_ptr, col):
    depth = np.ones(n, np.int64)
    for u in range(n):                      # tasks are topologically numbered
        for p in range(row_ptr[u], row_ptr[u + 1]):
            v = col[p]
            assert v > u
            depth[v] = max(depth[v], depth[u] + 1)
    return int(depth.max()) if n else 0


@pytest.mark.parametrize("T", [1, 2, 3, 8, 16, 32])
def test_cholesky_dag_closed_forms(T):
    tasks = O.cholesky_tasks(T, 64)
    t, k, m, _ = O.access_arrays(tasks)
    n = len(tasks)
    assert n == T + T * (T - 1) + T * (T - 1) * (T - 2) // 6
    row_ptr, col, deg = O.derive(n, t, k, m)
    assert len(col) == T * (T * T - 1) // 2
    assert longest_path(n, row_ptr, col) == 3 * T - 2
    # in-degree: POTRF 1, TRSM 2, SYRK 2, GEMM 3; one less at step k = 0
    for i, (op, acc, _) in enumerate(tasks):
        name = acc[0][0]                    # A_kk for POTRF/TRSM, A_ik for SYRK/GEMM
        step = name[1] if op in (O.POTRF, O.TRSM) else name[2]
        expect = {O.POTRF: 1, O.TRSM: 2, O.SYRK: 2, O.GEMM_NT_SUB: 3}[op] - (step == 0)
        assert deg[i] == expect, (i, op, acc)


def test_cholesky_solve_dag_counts():
    # T = 8: factorisation 120 tasks / 252 edges; solve adds T(T+1) = 72 tasks;
    # whole graph 192 tasks, 465 edges, critical path 38.
    tasks = O.cholesky_tasks(8, 64, with_solve=True)
    t, k, m, _ = O.access_arrays(tasks)
    row_ptr, col, _ = O.derive(len(tasks), t, k, m)
    assert len(tasks) == 192
    assert len(col) == 465
    assert longest_path(len(tasks), row_ptr, col) == 38


@pytest.mark.parametrize("T", [4, 16])
def test_gemm_dag_counts(T):
    tasks = O.gemm_tasks(T)
    t, k, m, _ = O.access_arrays(tasks)
    row_ptr, col, deg = O.derive(len(tasks), t, k, m)
    # T^2 independent chains of length T on the C blocks.
    assert len(tasks) == T ** 3
    assert len(col) == T * T * (T - 1)
    assert longest_path(len(tasks), row_ptr, col) == T
    # commutative: no edge at all (each C_ij is one run, A and B only read)
    tasks = O.gemm_tasks(T, commutative=True)
    t, k, m, _ = O.access_arrays(tasks)
    _, col, _ = O.derive(len(tasks), t, k, m)
    assert len(col) == 0


def merged(n, t, k, m):
    acc = [dict() for _ in range(n)]
    for ti, ki, mi in zip(t, k, m):
        d = acc[int(ti)]
        ki, mi = int(ki), int(mi)
        d[ki] = mi if ki not in d or d[ki] == mi else 1
    return acc


def conflict_closure(n, acc):
    """Brute-force STF order: u < v must be ordered when they share a key,
    unless both only read it, or both are commutative writes of the same run,
    or both are atomic writes of the same run (no access of another mode to
    that key between them).  A maybe-write (4) conflicts like a write."""
    need = np.zeros((n, n), bool)
    for u in range(n):
        for v in range(u + 1, n):
            for key in set(acc[u]) & set(acc[v]):
                a, b = acc[u][key], acc[v][key]
                if a == 0 and b == 0:
                    continue
                if a == b and a in (2, 3) and all(acc[w].get(key, a) == a
                                                  for w in range(u + 1, v)):
                    continue
                need[u, v] = True
    return closure(need)


def closure(adj):
    r = adj.copy()
    n = len(r)
    for w in range(n):
        r |= np.outer(r[:, w], r[w, :])
    return r


@pytest.mark.parametrize("seed", range(60))
def test_bruteforce_small_random(seed):
    n = 2 + seed % 9                         # 2..10 tasks
    t, k, m = inputs.random_access_lists(n, 1 + seed % 4, 4, seed=1000 + seed)
    ntask = int(t.max()) + 1
    row_ptr, col, deg = O.derive(ntask, t, k, m)
    adj = np.zeros((ntask, ntask), bool)
    for u, v in csr_edges(row_ptr, col):
        assert u < v
        adj[u, v] = True
    acc = merged(ntask, t, k, m)
    assert (closure(adj) == conflict_closure(ntask, acc)).all()
    assert (adj.sum(0) == deg).all()
    # no edge inside a READ group: such a pair never conflicts on any key it
    # shares, so an edge needs another shared key.
    for u, v in csr_edges(row_ptr, col):
        shared = set(acc[u]) & set(acc[v])
        assert shared
        assert any(not (acc[u][x] == 0 and acc[v][x] == 0) for x in shared)


@pytest.mark.parametrize("seed", range(60))
def test_bruteforce_small_random_five_modes(seed):
    """The same brute force with atomic and maybe writes in the lists."""
    n = 2 + seed % 9
    t, k, m = inputs.random_access_lists(n, 1 + seed % 4, 4, seed=3000 + seed, nmodes=5)
    ntask = int(t.max()) + 1
    row_ptr, col, deg = O.derive(ntask, t, k, m)
    adj = np.zeros((ntask, ntask), bool)
    for u, v in csr_edges(row_ptr, col):
        assert u < v
        adj[u, v] = True
    acc = merged(ntask, t, k, m)
    assert (closure(adj) == conflict_closure(ntask, acc)).all()
    assert (adj.sum(0) == deg).all()
    # no edge inside an atomic run: an edge needs a shared key on which the
    # pair is not two atomic writes
    for u, v in csr_edges(row_ptr, col):
        shared = set(acc[u]) & set(acc[v])
        assert any(not (acc[u][x] == 3 and acc[v][x] == 3) for x in shared)


def linear_extensions_ok(n, acc, adj):
    """Every order of the tasks that respects the edges gives each access the
    same view of its key as insertion order.  A key's state is its sequence of
    write segments: ("W", task) for a WRITE, a frozenset for a run of
    commutative writes (order inside the run does not matter).  A READ or
    WRITE sees the whole state; a commutative write sees the state before its
    run.  Interleaving anything inside a run splits the set and changes views."""
    def views(order):
        state = {}
        seen = {}
        for tsk in order:
            for key, md in acc[tsk].items():
                segs = state.setdefault(key, [])
                if md in (2, 3):   # a commutative or atomic run: a set
                    if segs and isinstance(segs[-1], tuple) and segs[-1][0] == md:
                        seen[(tsk, key)] = tuple(segs[:-1])
                        segs[-1] = (md, segs[-1][1] | {tsk})
                    else:
                        seen[(tsk, key)] = tuple(segs)
                        segs.append((md, frozenset([tsk])))
                else:
                    seen[(tsk, key)] = tuple(segs)
                    if md in (1, 4):   # a write, or a maybe-write
                        segs.append(("W", tsk))
        # the final state of every key must agree as well
        return seen, {k: tuple(v) for k, v in state.items()}
    ref = views(list(range(n)))
    pos = np.arange(n)
    for perm in itertools.permutations(range(n)):
        pos[list(perm)] = np.arange(n)
        if any(adj[u, v] and pos[u] > pos[v] for u in range(n) for v in range(n)):
            continue
        if views(list(perm)) != ref:
            return False
    return True


@pytest.mark.parametrize("seed", range(20))
def test_exhaustive_schedules(seed):
    n = 3 + seed % 5                         # 3..7 tasks
    t, k, m = inputs.random_access_lists(n, 2, 3, seed=7000 + seed,
                                         nmodes=3 if seed < 12 else 5)
    ntask = int(t.max()) + 1
    row_ptr, col, _ = O.derive(ntask, t, k, m)
    adj = np.zeros((ntask, ntask), bool)
    for u, v in csr_edges(row_ptr, col):
        adj[u, v] = True
    assert linear_extensions_ok(ntask, merged(ntask, t, k, m), adj)


def test_gemm_dag_atomic_counts():
    # ATOMIC_WRITE on C_ij: each block's tasks form one group, no edges
    tasks = O.gemm_tasks(4, mode=O.ATOMIC_WRITE)
    t, k, m, _ = O.access_arrays(tasks)
    _, col, _ = O.derive(len(tasks), t, k, m)
    assert len(col) == 0
    # MAYBE_WRITE orders like WRITE: the chains of the WRITE DAG
    tasks = O.gemm_tasks(4, mode=O.MAYBE_WRITE)
    t, k, m, _ = O.access_arrays(tasks)
    _, col, _ = O.derive(len(tasks), t, k, m)
    assert len(col) == 4 * 4 * 3


def test_merge_rule():
    # one task naming a key twice: R+R stays a read, R+C or R+W becomes a write
    for m2, expect_edge in ((0, False), (2, True), (1, True)):
        t = np.array([0, 1, 1, 2], np.uint32)
        k = np.array([0, 0, 0, 0], np.uint64)
        m = np.array([0, 0, m2, 0], np.int32)
        _, col, deg = O.derive(3, t, k, m)
        assert (deg[1] == 0) == (not expect_edge)
        assert (deg[2] == 1) == expect_edge


def test_malformed():
    with pytest.raises(ValueError):
        O.derive(2, np.array([1, 0], np.uint32), np.array([0, 0], np.uint64), np.array([0, 0], np.int32))
    with pytest.raises(ValueError):
        O.derive(1, np.array([0], np.uint32), np.array([0], np.uint64), np.array([5], np.int32))
    with pytest.raises(ValueError):
        O.derive(1, np.array([0], np.uint32), np.array([0], np.uint64), np.array([-1], np.int32))
