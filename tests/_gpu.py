"""Helpers shared by the GPU tests: run the product path through the C ABI."""
import numpy as np
import pytest
import torch


def need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def spx_mod():
    from paper_2308_15964_b300 import build
    build.build()
    from paper_2308_15964_b300 import spx
    return spx


def run_cholesky(A_np, b, X_np=None, lookahead=True, **cfg):
    """Tiled Cholesky (+ solve) of host arrays on the GPU; returns
    (status, info, L (full array, lower = factor), X, graph)."""
    from paper_2308_15964_b300 import cholesky
    S = spx_mod()
    A = torch.from_numpy(np.ascontiguousarray(A_np)).cuda()
    X = torch.from_numpy(np.ascontiguousarray(X_np)).cuda() if X_np is not None else None
    g = S.Graph(**cfg)
    cholesky.cholesky_graph(g, A, b, X, lookahead=lookahead)
    rc, info = g.run()
    torch.cuda.synchronize()
    return rc, info, A.cpu().numpy(), (X.cpu().numpy() if X is not None else None), g


def nop_graph(S, ntasks, task, key, mode, **cfg):
    """A graph of NOP tasks with the given access lists (keys map to fake,
    never dereferenced, tile addresses)."""
    g = S.Graph(**cfg)
    base = 0x7f0000000000
    handles = {}
    for k in np.unique(key):
        handles[int(k)] = g.register(base + 4096 * int(k), 8, 8, 8)
    t = 0
    i = 0
    while i < len(task):
        j = i
        while j < len(task) and task[j] == task[i]:
            j += 1
        assert task[i] == t
        g.insert(S.OP_NOP, [handles[int(k)] for k in key[i:j]], [int(m) for m in mode[i:j]])
        t += 1
        i = j
    assert t == ntasks
    return g
