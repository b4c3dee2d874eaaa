"""Host side of the batch driver, on the CPU: the seeded problem sizes and
the packing of many uneven problems into shared buffers (each on a 256-byte
boundary, none overlapping), including the split stores."""
import numpy as np
import pytest
import torch

from paper_2308_15964_b300 import batch, cholesky, inputs, spx


def test_problem_sizes_seeded_and_in_range():
    n, r = batch.problem_sizes(4096, seed=3)
    n2, r2 = batch.problem_sizes(4096, seed=3)
    assert np.array_equal(n, n2) and np.array_equal(r, r2)
    assert not np.array_equal(n, batch.problem_sizes(4096, seed=4)[0])
    assert n.min() >= 32 and n.max() <= 1024 and np.all(n % 32 == 0)
    assert r.min() >= 1 and r.max() <= 16
    # uniform over the 32 orders and the 16 widths: every value occurs
    assert len(np.unique(n)) == 32 and len(np.unique(r)) == 16


def _spans_disjoint(off, length):
    order = np.argsort(off)
    for a, b in zip(order, order[1:]):
        assert off[a] + length[a] <= off[b]


def test_batch_packing_and_views():
    n = np.array([32, 96, 64, 160, 40], np.int64)
    r = np.array([1, 3, 16, 2, 5], np.int64)
    B = batch.Batch(n, r, seed=5, device="cpu")
    assert np.all(B.a_off % 32 == 0) and np.all(B.x_off % 32 == 0)     # 32 doubles = 256 bytes
    _spans_disjoint(B.a_off, n * n)
    _spans_disjoint(B.x_off, n * r)
    for i in range(len(n)):
        k = int(n[i])
        assert torch.equal(B.a_view(i), inputs.spd_matrix(k, 1.0, B.seed_of(i), "cpu"))
        assert torch.equal(B.x_view(i), inputs.rhs(k, int(r[i]), B.seed_of(i), "cpu"))
        assert B.a_view(i).data_ptr() % 256 == B.A.data_ptr() % 256
    B.A.zero_()
    B.X.zero_()
    B.restore()
    assert torch.equal(B.a_view(3), inputs.spd_matrix(160, 1.0, B.seed_of(3), "cpu"))
    assert B.flops() == sum(cholesky.cholesky_flops(int(k), int(w)) for k, w in zip(n, r))


def test_split_buffers_sized_and_cached():
    n = np.array([128, 256, 96, 512], np.int64)
    B = batch.Batch(n, np.ones(4, np.int64), seed=1, device="cpu", fill=False)
    tiles = [64, 128, 32, 256]
    S, V = B.split_buffers(tiles)
    for i, (k, b) in enumerate(zip(n, tiles)):
        T = -(-int(k) // b)
        slot = spx.lib.spx_ozaki_slot_bytes(b)
        assert slot > 0 and slot % 256 == 0
        assert B.s_len[i] == (T * (T - 1) // 2 + T) * slot
        assert B.s_off[i] % 256 == 0 and B.v_off[i] % 32 == 0
    _spans_disjoint(B.s_off, B.s_len)
    _spans_disjoint(B.v_off, n * np.array(tiles))
    assert S.numel() == int(B.s_off[-1] + B.s_len[-1]) and S.dtype == torch.uint8
    assert V.numel() >= int(B.v_off[-1] + n[-1] * tiles[-1])
    S2, V2 = B.split_buffers(tiles)
    assert S2 is S and V2 is V                   # same tiles: the same buffers
    S3, _ = B.split_buffers([32, 32, 32, 32])
    assert S3 is not S


@pytest.mark.parametrize("b", [32, 64, 128, 256, 384, 512])
def test_slot_bytes_are_tma_aligned(b):
    # each split slot must start on a 256-byte boundary when packed back to back
    assert spx.lib.spx_ozaki_slot_bytes(b) % 256 == 0
