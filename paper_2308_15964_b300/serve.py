"""Serving loop: a Poisson stream of Cholesky-solve requests through the
continuous-batching server (spx_server_*).

Each request is one task graph: the tiled Cholesky of its matrix plus the
block solve of its right-hand sides, in FP64, or in mixed precision (TF32
tensor-core trailing updates) followed by FP64 refinement sweeps expressed as
tasks of the same graph (their correction solves apply the FP64 inverses of
the diagonal factor tiles, computed by TRTRI tasks of the graph).  Requests are admitted in arrival order (no
skipping) when their buffers fit in the HBM budget, an arena allocated once;
their inputs are staged into the arena by the copy engines (the resident
kernel holds the SMs).  Latency = completion time - arrival time (host wall
clock).
"""
from __future__ import annotations

import ctypes
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import cholesky, inputs, mixed, spx


@dataclass
class Request:
    idx: int
    arrival: float
    n: int
    nrhs: int
    prec: int
    tile: int
    bytes: int = 0
    offset: int = -1
    rid: int | None = None
    admitted: float = -1.0
    done: float = -1.0
    status: int = 0
    split: bool = False          # FP64 by split products on the tensor cores
    views: dict = field(default_factory=dict)


def request_stream(rate: float, duration: float, seed: int, nmin=64, nmax=16384, rhs_max=64,
                   tf32_frac=0.5):
    """Seeded Poisson arrivals; n log-uniform in [nmin, nmax] rounded to a
    multiple of 32; nrhs uniform in [1, rhs_max]; precision TF32 with
    probability tf32_frac, else FP64."""
    count = int(rate * duration * 2 + 100)
    u = inputs.uniform((4, count), seed).numpy() * 0.5 + 0.5     # [0, 1)
    gaps = -np.log(1.0 - u[0]) / rate
    t = np.cumsum(gaps)
    out = []
    for i in range(count):
        if t[i] > duration:
            break
        n = int(round(math.exp(math.log(nmin) + u[1, i] * (math.log(nmax) - math.log(nmin))) / 32) * 32)
        n = max(nmin, min(nmax, n))
        nrhs = 1 + int(u[2, i] * rhs_max)
        prec = spx.TF32 if u[3, i] < tf32_frac else spx.F64
        out.append(Request(i, float(t[i]), n, nrhs, prec, tile_for(n, prec)))
    return out


def tile_for(n: int, prec: int) -> int:
    if prec != spx.F64:
        return 256 if n <= 4096 else 512
    if n <= 256:
        return 64
    return 128 if n <= 2048 else (256 if n <= 8192 else 512)


# FP64 requests of at least this order run by split products (with split_fp64)
SPLIT_MIN_N = 2048


def split_store_bytes(n: int, b: int) -> int:
    """Split store of spx_cholesky_insert_ozaki with inverse panels."""
    T = -(-n // b)
    return (T * (T - 1) // 2 + T) * spx.lib.spx_ozaki_slot_bytes(b)


def request_bytes(n: int, nrhs: int, prec: int, split: bool = False) -> int:
    pad = lambda b: (b + 255) // 256 * 256
    if prec == spx.F64 and split:
        b = tile_for(n, prec)
        # A, X, the split store, V (the diagonal-tile inverses, n x b)
        return pad(8 * n * n) + pad(8 * n * nrhs) + pad(split_store_bytes(n, b)) + pad(8 * n * b)
    if prec == spx.F64:
        return pad(8 * n * n) + pad(8 * n * nrhs)
    # A (factored), A0 (original), A_lo (FP32 for TF32), V (diagonal-tile
    # inverses, n x tile), B, X, R, D
    return (2 * pad(8 * n * n) + pad(4 * n * n) + pad(8 * n * min(tile_for(n, prec), n)) +
            4 * pad(8 * n * nrhs))


class Arena:
    """First-fit sub-allocation of one device buffer (the HBM budget)."""

    def __init__(self, nbytes: int, device="cuda"):
        self.buf = torch.empty(nbytes // 8, dtype=torch.float64, device=device)
        self.free = [(0, nbytes)]

    def alloc(self, nbytes):
        for k, (o, ln) in enumerate(self.free):
            if ln >= nbytes:
                if ln == nbytes:
                    self.free.pop(k)
                else:
                    self.free[k] = (o + nbytes, ln - nbytes)
                return o
        return -1

    def release(self, o, nbytes):
        self.free.append((o, nbytes))
        self.free.sort()
        merged = []
        for a, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((a, ln))
        self.free = merged

    def view(self, off, shape, dtype=torch.float64):
        elems = int(np.prod(shape))
        es = torch.tensor([], dtype=dtype).element_size()
        base = self.buf.view(torch.uint8)[off:off + elems * es]
        return base.view(dtype).view(*shape)


class Sources:
    """Request inputs: leading blocks of one SPD matrix of the largest order
    (A = B B^T / N + I, principal submatrices are SPD) and of one RHS block."""

    def __init__(self, nmax: int, rhs_max: int, seed: int):
        self.A = inputs.spd_matrix(nmax, 1.0, seed, device="cuda")
        self.B = inputs.rhs(nmax, rhs_max, seed, device="cuda")
        torch.cuda.synchronize()

    def stage(self, dst, src, rows, cols, stream):
        """Copy-engine copy of src[:rows, :cols] into the contiguous dst."""
        spx._check(spx.lib.spx_copy2d(ctypes.c_void_p(dst.data_ptr()), cols * 8,
                                      ctypes.c_void_p(src.data_ptr()), src.stride(0) * 8, cols * 8,
                                      rows, ctypes.c_void_p(stream.cuda_stream)), "spx_copy2d")


def build_graph(req: Request, arena: Arena, src: Sources, stream, sweeps: int = 4):
    n, r = req.n, req.nrhs
    pad = lambda b: (b + 255) // 256 * 256
    o = req.offset
    A = arena.view(o, (n, n))
    o += pad(8 * n * n)
    g = spx.Graph()
    if req.prec == spx.F64:
        X = arena.view(o, (n, r))
        o += pad(8 * n * r)
        src.stage(A, src.A, n, n, stream)
        src.stage(X, src.B, n, r, stream)
        stream.synchronize()
        if req.split:
            sb = split_store_bytes(n, req.tile)
            S = arena.view(o, (sb,), torch.uint8)
            o += pad(sb)
            V = arena.view(o, (n, req.tile))
            cholesky.cholesky_ozaki_graph(g, A, req.tile, X, S=S, V=V)
        else:
            cholesky.cholesky_graph(g, A, req.tile, X)
        req.views = {"A": A, "X": X}
        return g
    A0 = arena.view(o, (n, n))
    o += pad(8 * n * n)
    Alo = arena.view(o, (n, n), torch.float32)
    o += pad(4 * n * n)
    B = arena.view(o, (n, r))
    o += pad(8 * n * r)
    X = arena.view(o, (n, r))
    o += pad(8 * n * r)
    R = arena.view(o, (n, r))
    o += pad(8 * n * r)
    D = arena.view(o, (n, r))
    o += pad(8 * n * r)
    vb = min(req.tile, n)
    V = arena.view(o, (n, vb))
    for dst, s_, rows, cols in ((A, src.A, n, n), (A0, src.A, n, n), (B, src.B, n, r), (X, src.B, n, r)):
        src.stage(dst, s_, rows, cols, stream)
    stream.synchronize()
    mixed.factor_graph(g, A, Alo, req.tile, X, req.prec)
    nt = ctypes.c_longlong()
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    spx._check(spx.lib.spx_refine_inv_insert(g._h, P(A0), n, n, P(A), n, req.tile, P(V), vb, P(B),
                                             P(X), P(R), P(D), r, r, sweeps, ctypes.byref(nt)),
               "spx_refine_inv_insert")
    req.views = {"A": A, "A0": A0, "B": B, "X": X}
    return g


def serve(rate=200.0, duration=60.0, budget=120e9, seed=6, nmax=16384, rhs_max=64, tf32_frac=0.5,
          sweeps=4, drain=True, max_wall=None, keep_results=False, split_fp64=False):
    """Run the stream; returns a summary dict (and the finished requests).
    split_fp64: FP64 requests of order >= SPLIT_MIN_N run by split products
    on the tensor cores (the server's one-CTA-per-SM kernel), FP64 results."""
    reqs = request_stream(rate, duration, seed, nmax=nmax, rhs_max=rhs_max, tf32_frac=tf32_frac)
    src = Sources(nmax, rhs_max, seed)
    arena = Arena(int(budget))
    srv = spx.Server(tensor_cores=2 if split_fp64 else 1, idle_ns=200_000_000)
    stream = torch.cuda.Stream()
    for q in reqs:
        q.split = split_fp64 and q.prec == spx.F64 and q.n >= SPLIT_MIN_N
        q.bytes = request_bytes(q.n, q.nrhs, q.prec, q.split)
    pending = list(reqs)
    live, finished = [], []
    t0 = time.perf_counter()
    max_wall = max_wall or (duration * 10 + 60)
    while pending or live:
        now = time.perf_counter() - t0
        if now > max_wall:
            break
        # admit in arrival order while the budget allows (no skipping)
        while pending and pending[0].arrival <= now and (drain or now <= duration):
            q = pending[0]
            q.offset = arena.alloc(q.bytes)
            if q.offset < 0:
                break
            g = build_graph(q, arena, src, stream, sweeps)
            rid = srv.submit(g)
            g.close()
            if rid is None:                       # server pools full: retry later
                arena.release(q.offset, q.bytes)
                q.offset = -1
                break
            q.rid, q.admitted = rid, time.perf_counter() - t0
            live.append(pending.pop(0))
        if not drain and now > duration:
            pending = []
        still = []
        for q in live:
            res = srv.poll(q.rid)
            if res is None:
                still.append(q)
                continue
            q.done = time.perf_counter() - t0
            q.status = res[0]
            if not keep_results:
                arena.release(q.offset, q.bytes)
            finished.append(q)
        live = still
        if not pending and not live:
            break
        time.sleep(0.0002)
    wall = time.perf_counter() - t0
    srv.stop()
    srv.close()
    lat = np.array([q.done - q.arrival for q in finished]) if finished else np.zeros(1)
    flops = sum(cholesky.cholesky_flops(q.n, q.nrhs) for q in finished)
    out = {
        "offered_rate": rate, "duration_s": duration, "budget_gb": budget / 1e9,
        "requests": len(reqs), "completed": len(finished),
        "failed": sum(1 for q in finished if q.status != 0),
        "backlog_at_end": len(reqs) - len(finished),
        "wall_s": wall, "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "throughput_req_s": len(finished) / wall, "gflops": flops / wall / 1e9,
        "tf32_requests": sum(1 for q in finished if q.prec != spx.F64),
        "split_fp64_requests": sum(1 for q in finished if q.split),
    }
    return (out, finished, arena) if keep_results else out
