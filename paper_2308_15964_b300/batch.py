"""Batched uneven Cholesky solves in one persistent launch, and the tile
autotuner.

Thousands of independent SPD systems A_i X_i = B_i of different orders are
inserted into ONE task graph (spx_cholesky_insert_batch).  They share no tile,
so their DAGs are disjoint and a single persistent launch interleaves all of
their tasks.  Each problem's tile comes from an autotuner that times the
candidate tiles on the GPU.  Re-running the same batch shape (new values in the
same buffers) replays one CUDA graph (cfg.cuda_graph).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import cholesky, inputs, spx

TILES = (32, 64, 128, 256)


def problem_sizes(count: int, seed: int, nmax: int = 1024, rhs_max: int = 16):
    """n_i uniform on the multiples of 32 in [32, nmax]; nrhs_i uniform in [1, rhs_max]."""
    x = inputs.splitmix64(torch.arange(0, 2 * count, dtype=torch.int64), seed).numpy().view(np.uint64)
    n = 32 * (1 + (x[:count] % np.uint64(nmax // 32)).astype(np.int64))
    r = 1 + (x[count:] % np.uint64(rhs_max)).astype(np.int64)
    return n.astype(np.int64), r.astype(np.int64)


class Batch:
    """Packed device buffers of a batch: A_i (n_i x n_i) and X_i (n_i x nrhs_i)
    back to back, each starting on a 256-byte boundary."""

    def __init__(self, n, nrhs, seed: int, device="cuda", sigma: float = 1.0, fill: bool = True):
        self.n = np.asarray(n, np.int64)
        self.nrhs = np.asarray(nrhs, np.int64)
        self.count = len(self.n)
        pad = lambda e: (e + 31) // 32 * 32          # 32 doubles = 256 bytes
        a_sz = [pad(int(k) * int(k)) for k in self.n]
        x_sz = [pad(int(k) * int(r)) for k, r in zip(self.n, self.nrhs)]
        self.a_off = np.concatenate([[0], np.cumsum(a_sz)[:-1]]).astype(np.int64)
        self.x_off = np.concatenate([[0], np.cumsum(x_sz)[:-1]]).astype(np.int64)
        self.A = torch.empty(int(sum(a_sz)), dtype=torch.float64, device=device)
        self.X = torch.empty(int(sum(x_sz)), dtype=torch.float64, device=device)
        self.seed = seed
        self.sigma = sigma
        if fill:
            for i in range(self.count):
                self.a_view(i).copy_(inputs.spd_matrix(int(self.n[i]), sigma, self.seed_of(i), device))
                self.x_view(i).copy_(inputs.rhs(int(self.n[i]), int(self.nrhs[i]), self.seed_of(i), device))
        self.A0 = self.A.clone() if fill else None
        self.X0 = self.X.clone() if fill else None

    def seed_of(self, i: int) -> int:
        return self.seed * (1 << 32) + i

    def a_view(self, i):
        k = int(self.n[i])
        return self.A[int(self.a_off[i]):int(self.a_off[i]) + k * k].view(k, k)

    def x_view(self, i):
        k, r = int(self.n[i]), int(self.nrhs[i])
        return self.X[int(self.x_off[i]):int(self.x_off[i]) + k * r].view(k, r)

    def restore(self):
        self.A.copy_(self.A0)
        self.X.copy_(self.X0)

    def flops(self) -> float:
        return float(sum(cholesky.cholesky_flops(int(k), int(r)) for k, r in zip(self.n, self.nrhs)))


def insert(g: spx.Graph, batch: Batch, tiles, lookahead: bool = False) -> int:
    """Insert every problem of the batch; tiles[i] is problem i's tile.  By
    default without look-ahead priorities: thousands of independent problems
    keep every SM busy, so critical-path splitting (finer parts, more queue
    traffic) only costs throughput (measured: 842 vs 860 GFLOP/s on the
    4096-problem batch)."""
    c = batch.count
    base_a, base_x = batch.A.data_ptr(), batch.X.data_ptr()
    pa = (ctypes.c_void_p * c)(*[base_a + 8 * int(o) for o in batch.a_off])
    px = (ctypes.c_void_p * c)(*[base_x + 8 * int(o) for o in batch.x_off])
    n = np.ascontiguousarray(batch.n, np.int32)
    b = np.ascontiguousarray(tiles, np.int32)
    r = np.ascontiguousarray(batch.nrhs, np.int32)
    nt = ctypes.c_longlong()
    ip = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    spx._check(spx.lib.spx_cholesky_insert_batch(g._h, c, pa, ip(n), ip(n), ip(b), px, ip(r), ip(r),
                                                 1 if lookahead else 0, spx.F64, ctypes.byref(nt)),
               "spx_cholesky_insert_batch")
    g._keep.append(batch)
    return nt.value


def autotune(sizes, copies: int = 148, candidates=TILES, seed: int = 99):
    """Pick, for every distinct n, the tile with the shortest persistent-kernel
    time on a batch of `copies` problems of that order (one matrix replicated).
    Candidates larger than n collapse to one tile, so only the smallest of
    them is tried.  Returns ({n: tile}, {n: {tile: ms}})."""
    best, table = {}, {}
    for k in sorted(set(int(s) for s in sizes)):
        cands = [b for b in candidates if b < k] + [min([b for b in candidates if b >= k] or [k])]
        bt = Batch([k] * copies, [1] * copies, seed, fill=False)
        a = inputs.spd_matrix(k, 1.0, seed)
        a_dev = a.cuda()
        times = {}
        for b in cands:
            for i in range(copies):
                bt.a_view(i).copy_(a_dev)
            bt.X.fill_(1.0)
            g = spx.Graph(cuda_graph=True)
            insert(g, bt, [b] * copies)
            rc, _ = g.run()
            assert rc == spx.OK, rc
            g.reset()
            for i in range(copies):
                bt.a_view(i).copy_(a_dev)
            bt.X.fill_(1.0)
            rc, _ = g.run()
            assert rc == spx.OK, rc
            times[b] = g.timing()[1]
            g.close()
        table[k] = times
        best[k] = min(times, key=times.get)
    return best, table
