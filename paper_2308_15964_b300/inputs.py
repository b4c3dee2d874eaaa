"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the method itself: it only draws random
numbers and forms the synthetic SPD matrices, right-hand sides and access
lists that both sides consume.  Every value is defined bit-for-bit, so the
same call on the CPU and on the GPU returns identical bytes.

Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: the i-th draw of stream ``seed`` is ``mix(seed + (i+1)*GOLDEN)``.

SPD matrices follow the workload of the paper's tiled Cholesky experiments:
``A = B B^T / n + sigma I`` with ``B`` entries uniform on [-1, 1].  To make the
product exact on any device, ``B`` is drawn from the 255-level lattice
``k/127`` with ``k`` uniform on the integers -127..127.  ``G = K K^T`` is then an
integer matrix: every partial sum of 512 products stays below 2^24, so an
FP32 (or TF32) GEMM over 512-column slices is exact, and so is the FP64
accumulation of the slices.  ``A = G / (127^2 n)`` (one correctly rounded
division) plus ``sigma`` on the diagonal.
"""
from __future__ import annotations

import math

import numpy as np
import torch

GOLDEN = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_KMAX = 127          # B entries are k / 127, k in [-127, 127]
_SLICE = 512         # column slice for the exact FP32 product


def _s64(x: int) -> int:
    """Python int modulo 2^64 reinterpreted as signed int64."""
    x &= (1 << 64) - 1
    return x - (1 << 64) if x >= (1 << 63) else x


def _lsr(z: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def splitmix64(counter: torch.Tensor, seed: int) -> torch.Tensor:
    """Raw 64-bit splitmix64 outputs (as int64 bit patterns) for int64 counters."""
    z = counter * _s64(GOLDEN) + _s64(seed + GOLDEN)
    z = (z ^ _lsr(z, 30)) * _s64(_M1)
    z = (z ^ _lsr(z, 27)) * _s64(_M2)
    return z ^ _lsr(z, 31)


def splitmix64_ref(seed: int, i: int) -> int:
    """Scalar Python reference of the i-th draw (unsigned), for tests."""
    z = (seed + (i + 1) * GOLDEN) & ((1 << 64) - 1)
    z = ((z ^ (z >> 30)) * _M1) & ((1 << 64) - 1)
    z = ((z ^ (z >> 27)) * _M2) & ((1 << 64) - 1)
    return z ^ (z >> 31)


def _counters(start: int, count: int, device) -> torch.Tensor:
    return torch.arange(start, start + count, dtype=torch.int64, device=device)


def uniform(shape, seed: int, device="cpu", start: int = 0) -> torch.Tensor:
    """FP64 uniform on [-1, 1): u = ((x >> 11) * 2^-53) * 2 - 1 (exact)."""
    count = int(np.prod(shape)) if len(shape) else 1
    x = splitmix64(_counters(start, count, device), seed)
    u = _lsr(x, 11).to(torch.float64) * (2.0 ** -53)
    return (u * 2.0 - 1.0).reshape(shape)


def int_lattice(rows: int, cols: int, seed: int, device="cpu", col0: int = 0,
                ncols_total: int | None = None) -> torch.Tensor:
    """Integers k in [-127, 127] (int64), entry (i, j) from counter i*ncols_total + col0 + j."""
    total = cols if ncols_total is None else ncols_total
    i = torch.arange(rows, dtype=torch.int64, device=device).unsqueeze(1)
    j = torch.arange(col0, col0 + cols, dtype=torch.int64, device=device).unsqueeze(0)
    x = splitmix64(i * total + j, seed)
    return ((_lsr(x, 32) * (2 * _KMAX + 1)) >> 32) - _KMAX


def spd_matrix(n: int, sigma: float, seed: int, device="cpu") -> torch.Tensor:
    """A = B B^T / n + sigma I, exactly symmetric, identical bytes on any device.

    Row-major n x n FP64.  CPU: FP64 product of integer-valued matrices (exact,
    all partial sums < 2^53).  CUDA: FP32 products of 512-column slices (exact,
    partial sums < 2^24) accumulated in FP64 (exact).
    """
    dev = torch.device(device)
    g = torch.zeros((n, n), dtype=torch.float64, device=dev)
    for c0 in range(0, n, _SLICE):
        c1 = min(n, c0 + _SLICE)
        k = int_lattice(n, c1 - c0, seed, dev, col0=c0, ncols_total=n)
        if dev.type == "cuda":
            kf = k.to(torch.float32)
            g += (kf @ kf.T).to(torch.float64)
            del kf
        else:
            kd = k.to(torch.float64)
            g += kd @ kd.T
        del k
    a = g.div_(float(_KMAX * _KMAX * n))
    a.diagonal().add_(sigma)
    return a


def rhs(n: int, nrhs: int, seed: int, device="cpu") -> torch.Tensor:
    """Right-hand sides, n x nrhs row-major, uniform on [-1, 1)."""
    return uniform((n, nrhs), seed ^ 0x5DEECE66D, device)


def gaussian(n: int, seed: int) -> np.ndarray:
    """Standard normal vector (Box-Muller on splitmix64 uniforms), CPU only."""
    m = (n + 1) // 2
    x = splitmix64(_counters(0, 2 * m, "cpu"), seed)
    u = (_lsr(x, 11).to(torch.float64) + 0.5) * (2.0 ** -53)
    u1, u2 = u[:m].numpy(), u[m:].numpy()
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * math.pi * u2), r * np.sin(2 * math.pi * u2)])
    return z[:n].copy()


def random_access_lists(ntasks: int, nkeys: int, max_handles: int, seed: int,
                        allow_repeats: bool = True, nmodes: int = 3):
    """Random STF access lists: per task 1..max_handles accesses on keys 0..nkeys-1.

    Returns (task, key, mode) int arrays in insertion order.  Modes are drawn
    from the first nmodes of 0 = READ, 1 = WRITE, 2 = COMMUTATIVE_WRITE,
    3 = ATOMIC_WRITE, 4 = MAYBE_WRITE.  Keys may repeat inside a task when
    allow_repeats is set (the merge rule is then exercised).
    """
    x = splitmix64(_counters(0, ntasks * (1 + 3 * max_handles), "cpu"), seed).numpy()
    x = x.view(np.uint64)
    pos = 0
    tasks, keys, modes = [], [], []
    for t in range(ntasks):
        nh = 1 + int(x[pos] % np.uint64(max_handles))
        pos += 1
        used = set()
        for _ in range(nh):
            k = int(x[pos] % np.uint64(nkeys))
            m = int(x[pos + 1] % np.uint64(nmodes))
            pos += 3
            if not allow_repeats and k in used:
                continue
            used.add(k)
            tasks.append(t)
            keys.append(k)
            modes.append(m)
    return (np.asarray(tasks, dtype=np.uint32), np.asarray(keys, dtype=np.uint64),
            np.asarray(modes, dtype=np.int32))
