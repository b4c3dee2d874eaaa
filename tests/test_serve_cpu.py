"""Host side of the serving driver, on the CPU: the first-fit arena that
holds the HBM budget, the seeded request stream and the per-request byte
accounting that admission relies on."""
import math

import numpy as np
import pytest

from paper_2308_15964_b300 import serve, spx


def _check_arena(arena, live, total):
    """Free list sorted, merged and disjoint; free + live bytes = total; no
    live block overlaps another or a free one."""
    free = arena.free
    assert free == sorted(free)
    for (a, la), (b, _) in zip(free, free[1:]):
        assert a + la < b                        # merged: no touching free blocks
    spans = sorted([(o, ln) for o, ln in free] + list(live.values()))
    pos = 0
    for o, ln in spans:
        assert o == pos and ln > 0
        pos = o + ln
    assert pos == total


def test_arena_first_fit_and_merge():
    total = 1 << 16
    a = serve.Arena(total, device="cpu")
    x = a.alloc(4096)
    y = a.alloc(8192)
    z = a.alloc(4096)
    assert (x, y, z) == (0, 4096, 12288)
    a.release(y, 8192)
    assert a.alloc(16384) == 16384               # the hole is too small: first fit after z
    assert a.alloc(8192) == 4096                 # the hole, exactly
    a.release(x, 4096)
    a.release(4096, 8192)
    a.release(z, 4096)
    a.release(16384, 16384)
    assert a.free == [(0, total)]
    assert a.alloc(total + 8) == -1


def test_arena_random_sequence_against_occupancy():
    rng = np.random.default_rng(7)
    total = 1 << 14
    a = serve.Arena(total, device="cpu")
    live = {}
    for step in range(2000):
        if live and (rng.random() < 0.45 or len(live) > 40):
            k = list(live)[rng.integers(len(live))]
            a.release(*live.pop(k))
        else:
            n = int(rng.integers(1, 64)) * 8
            o = a.alloc(n)
            if o < 0:
                # first fit failed: no free block is large enough
                assert all(ln < n for _, ln in a.free)
                continue
            live[step] = (o, n)
        _check_arena(a, live, total)


def test_arena_view_is_the_sub_buffer():
    import torch
    a = serve.Arena(4096, device="cpu")
    a.buf.zero_()
    o = a.alloc(1024)
    v = a.view(o, (4, 8))
    v.fill_(3.0)
    w = a.view(o + 256, (32,), dtype=torch.float32)
    assert w.numel() == 32 and float(a.buf[o // 8]) == 3.0
    assert float(a.buf.sum()) == 3.0 * 32


def test_request_stream_is_seeded_poisson():
    r1 = serve.request_stream(50.0, 40.0, seed=6)
    r2 = serve.request_stream(50.0, 40.0, seed=6)
    assert [(q.arrival, q.n, q.nrhs, q.prec) for q in r1] == \
        [(q.arrival, q.n, q.nrhs, q.prec) for q in r2]
    t = np.array([q.arrival for q in r1])
    assert np.all(np.diff(t) > 0) and t[-1] <= 40.0
    # 2000 expected arrivals: the count is within 4 standard deviations
    assert abs(len(r1) - 2000) < 4 * math.sqrt(2000)
    for q in r1:
        assert 64 <= q.n <= 16384 and q.n % 32 == 0
        assert 1 <= q.nrhs <= 64
        assert q.prec in (spx.TF32, spx.F64)
        assert q.tile == serve.tile_for(q.n, q.prec)
    frac = np.mean([q.prec == spx.TF32 for q in r1])
    assert abs(frac - 0.5) < 0.05
    # log-uniform orders: about half below the geometric mean of the range
    below = np.mean([q.n < math.sqrt(64 * 16384) for q in r1])
    assert abs(below - 0.5) < 0.05


@pytest.mark.parametrize("n,prec,tile", [(64, "F64", 64), (256, "F64", 64), (288, "F64", 128),
                                         (2048, "F64", 128), (2080, "F64", 256),
                                         (8192, "F64", 256), (8224, "F64", 512),
                                         (4096, "TF32", 256), (4128, "TF32", 512)])
def test_tile_for(n, prec, tile):
    assert serve.tile_for(n, getattr(spx, prec)) == tile


def test_request_bytes():
    pad = lambda b: -(-b // 256) * 256
    n, r = 1000, 7
    assert serve.request_bytes(n, r, spx.F64) == pad(8 * n * n) + pad(8 * n * r)
    b = serve.tile_for(n, spx.TF32)
    assert serve.request_bytes(n, r, spx.TF32) == \
        2 * pad(8 * n * n) + pad(4 * n * n) + pad(8 * n * min(b, n)) + 4 * pad(8 * n * r)
    n = 4096
    b = serve.tile_for(n, spx.F64)
    T = -(-n // b)
    slots = T * (T - 1) // 2 + T                 # lower tiles below the diagonal + V
    store = slots * spx.lib.spx_ozaki_slot_bytes(b)
    assert serve.split_store_bytes(n, b) == store
    assert serve.request_bytes(n, r, spx.F64, split=True) == \
        pad(8 * n * n) + pad(8 * n * r) + pad(store) + pad(8 * n * b)
    # every byte count is a multiple of the arena's 256-byte alignment
    for prec, split in ((spx.F64, False), (spx.F64, True), (spx.TF32, False)):
        assert serve.request_bytes(3000, 5, prec, split) % 256 == 0
