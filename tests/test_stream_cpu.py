"""Host-side derivation of a stream (spx_graph_host_preds) against the
oracle's DAG: the same edge set as the device derivation, transposed to
predecessor lists, on random access lists (three and five modes, repeated
handles in a task) and on the tiled Cholesky + solve task list.  No device
work (the tiles are fake addresses)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2308_15964_b300 import inputs
from tests._gpu import nop_graph


def spx():
    from paper_2308_15964_b300 import build
    build.build()
    from paper_2308_15964_b300 import spx as S
    return S


def oracle_preds(ntasks, task, key, mode):
    rp, col, _ = O.derive(ntasks, task, key, mode)
    preds = [[] for _ in range(ntasks)]
    for u in range(ntasks):
        for v in col[rp[u]:rp[u + 1]]:
            preds[int(v)].append(u)
    return [sorted(p) for p in preds]


def host_preds(g):
    ptr, pred = g.host_preds()
    return [sorted(pred[ptr[v]:ptr[v + 1]].tolist()) for v in range(len(ptr) - 1)]


@pytest.mark.parametrize("seed,nmodes", [(s, 3) for s in range(6)] + [(s, 5) for s in range(6)])
def test_host_preds_random_lists(seed, nmodes):
    S = spx()
    ntasks = 300 + 50 * seed
    task, key, mode = inputs.random_access_lists(ntasks, 12 + seed, 4, seed, nmodes=nmodes)
    g = nop_graph(S, ntasks, task, key, mode)
    assert host_preds(g) == oracle_preds(ntasks, task, key, mode)
    g.close()


@pytest.mark.parametrize("T,with_solve", [(1, False), (5, True), (8, False), (12, True)])
def test_host_preds_cholesky(T, with_solve):
    S = spx()
    tasks = O.cholesky_tasks(T, 64, with_solve=with_solve)
    task, key, mode = O.access_arrays(tasks)[:3]
    n = len(tasks)
    g = nop_graph(S, n, task, key, mode)
    assert host_preds(g) == oracle_preds(n, task, key, mode)
    g.close()
