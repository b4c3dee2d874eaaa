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

    def split_buffers(self, tiles):
        """Per-problem split stores (spx_cholesky_insert_ozaki with inverse
        panels: T (T - 1) / 2 + T slots) and diagonal-inverse blocks V_i
        (n_i x b_i), packed on 256-byte boundaries; kept for the tile choice."""
        key = tuple(int(t) for t in tiles)
        if getattr(self, "_split_key", None) != key:
            s_sz, v_sz = [], []
            for k, b in zip(self.n, key):
                T = -(-int(k) // b)
                s_sz.append((T * (T - 1) // 2 + T) * spx.lib.spx_ozaki_slot_bytes(b))
                v_sz.append((int(k) * b + 31) // 32 * 32)
            self.s_off = np.concatenate([[0], np.cumsum(s_sz)[:-1]]).astype(np.int64)
            self.s_len = np.asarray(s_sz, np.int64)
            self.v_off = np.concatenate([[0], np.cumsum(v_sz)[:-1]]).astype(np.int64)
            self.S = torch.empty(int(sum(s_sz)), dtype=torch.uint8, device=self.A.device)
            self.V = torch.empty(int(sum(v_sz)), dtype=torch.float64, device=self.A.device)
            self._split_key = key
        return self.S, self.V


def insert(g: spx.Graph, batch: Batch, tiles, lookahead: bool = False, split: bool = False) -> int:
    """Insert every problem of the batch; tiles[i] is problem i's tile.  By
    default without look-ahead priorities: thousands of independent problems
    keep every SM busy, so critical-path splitting (finer parts, more queue
    traffic) only costs throughput (measured: 842 vs 860 GFLOP/s on the
    4096-problem batch).  split: every problem by spx_cholesky_insert_ozaki
    (trailing updates and inverse panel products split on the tensor cores,
    FP64 results; tiles multiples of 32), with the stores of split_buffers."""
    c = batch.count
    if split:
        S, V = batch.split_buffers(tiles)
        total, nt = 0, ctypes.c_longlong()
        for i in range(c):
            k, b, r = int(batch.n[i]), int(tiles[i]), int(batch.nrhs[i])
            spx._check(spx.lib.spx_cholesky_insert_ozaki(
                g._h, ctypes.c_void_p(batch.A.data_ptr() + 8 * int(batch.a_off[i])), k, k, b,
                ctypes.c_void_p(S.data_ptr() + int(batch.s_off[i])), int(batch.s_len[i]),
                ctypes.c_void_p(V.data_ptr() + 8 * int(batch.v_off[i])), b, 0,
                ctypes.c_void_p(batch.X.data_ptr() + 8 * int(batch.x_off[i])), r, r,
                1 if lookahead else 0, ctypes.byref(nt)), "spx_cholesky_insert_ozaki")
            total += nt.value
        g._keep.append(batch)
        return total
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


def autotune(sizes, copies: int = 148, candidates=TILES, seed: int = 99, split: bool = False):
    """Pick, for every distinct n, the tile with the shortest persistent-kernel
    time on a batch of `copies` problems of that order (one matrix replicated).
    Candidates larger than n collapse to one tile, so only the smallest of
    them is tried.  split: time the split-product form (insert(split=True)).
    Returns ({n: tile}, {n: {tile: ms}})."""
    best, table = {}, {}
    for k in sorted(set(int(s) for s in sizes)):
        cands = [b for b in candidates if b < k] + [min([b for b in candidates if b >= k] or [k])]
        if split:  # split slots hold tiles of at most 512
            cands = [b for b in cands if b <= 512]
        bt = Batch([k] * copies, [1] * copies, seed, fill=False)
        a = inputs.spd_matrix(k, 1.0, seed)
        a_dev = a.cuda()
        times = {}
        for b in cands:
            for i in range(copies):
                bt.a_view(i).copy_(a_dev)
            bt.X.fill_(1.0)
            g = spx.Graph(cuda_graph=True)
            insert(g, bt, [b] * copies, split=split)
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
