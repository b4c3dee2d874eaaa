"""Streaming STF on the GPU: tasks inserted while the persistent kernel runs
(spx_stream_begin / spx_stream_flush / spx_stream_end).

* the tiled Cholesky inserted panel by panel, each panel flushed while the
  earlier ones run: the factor is bit-identical to the one-shot graph's (the
  same tile operations on the same data, in an order the dependencies fix);
* random access lists (three and five modes) inserted in batches of NOP
  tasks: every edge of the oracle's DAG is respected by the execution
  tickets (end of the predecessor before the start of the successor) and
  every task ran;
* a writer followed by 300 readers and a writer: the first writer's 300
  successors overflow its 64 successor slots, so relays are appended; the
  order is still the STF order;
* errors: insertion beyond the capacity, calls after the end.
"""
import time

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2308_15964_b300 import inputs
from tests._gpu import need_cuda, run_cholesky, spx_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    need_cuda()
    return spx_mod()


def insert_cholesky_panel(S, g, h, T, b, k, n):
    """The tasks of panel k of the tiled Cholesky (insertion order and
    priorities of spx_cholesky_insert with look-ahead)."""
    R, W = S.READ, S.WRITE
    t = g.insert(S.OP_POTRF, [h[k][k]], [W], 2)
    g.set_arg(t, k * b)
    for i in range(k + 1, T):
        g.insert(S.OP_TRSM, [h[k][k], h[i][k]], [R, W], 2 if i == k + 1 else 1)
    for i in range(k + 1, T):
        g.insert(S.OP_SYRK, [h[i][k], h[i][i]], [R, W], 2 if i == k + 1 else 1)
    for j in range(k + 1, T):
        for i in range(j + 1, T):
            g.insert(S.OP_GEMM_NT_SUB, [h[i][k], h[j][k], h[i][j]], [R, R, W],
                     (2 if i == k + 2 else 1) if j == k + 1 else 0)


@pytest.mark.parametrize("n,b,pause", [(1024, 128, 0.002), (2048, 256, 0.0), (1000, 128, 0.01)])
def test_stream_cholesky_bit_identical(S, n, b, pause):
    A = inputs.spd_matrix(n, 1.0, seed=n).numpy()
    rc, info, Lref, _, g0 = run_cholesky(A, b)
    assert rc == 0 and info == 0
    g0.close()
    Ad = torch.from_numpy(A.copy()).cuda()
    T = -(-n // b)
    g = S.Graph()
    h = [[None] * T for _ in range(T)]
    for i in range(T):
        for j in range(i + 1):
            r, c = min(b, n - i * b), min(b, n - j * b)
            h[i][j] = g.register(Ad[i * b:, j * b:].data_ptr(), r, c, n)
    g.stream_begin(max_tasks=4096, max_tiles=T * T, max_records=16384, max_preds=32768)
    for k in range(T):
        insert_cholesky_panel(S, g, h, T, b, k, n)
        g.stream_flush()
        if pause:
            time.sleep(pause)
    g.stream_end()
    rc, info = g.wait()
    assert rc == 0 and info == 0
    torch.cuda.synchronize()
    assert np.array_equal(np.tril(Ad.cpu().numpy()), np.tril(Lref))
    g.close()


@pytest.mark.parametrize("seed,nmodes,batch", [(1, 3, 100), (2, 5, 37), (3, 3, 1), (4, 5, 500)])
def test_stream_random_lists_tickets(S, seed, nmodes, batch):
    ntasks = 1500
    task, key, mode = inputs.random_access_lists(ntasks, 24, 4, seed, nmodes=nmodes)
    rp, col, _ = O.derive(ntasks, task, key, mode)
    g = S.Graph()
    base = 0x7f0000000000
    handles = {int(k): g.register(base + 4096 * int(k), 8, 8, 8) for k in np.unique(key)}
    g.stream_begin(max_tasks=4 * ntasks, max_tiles=64, max_records=8 * ntasks,
                   max_preds=64 * ntasks)
    ids = []
    i = 0
    for t in range(ntasks):
        j = i
        while j < len(task) and task[j] == t:
            j += 1
        ids.append(g.insert(S.OP_NOP, [handles[int(k)] for k in key[i:j]],
                            [int(m) for m in mode[i:j]]))
        i = j
        if (t + 1) % batch == 0:
            g.stream_flush()
    g.stream_end()
    rc, _ = g.wait()
    assert rc == 0
    s, e = g.tickets()
    ids = np.asarray(ids)
    assert (e[ids] > 0).all() and (s[ids] != 0xFFFFFFFF).all()
    for u in range(ntasks):
        for v in col[rp[u]:rp[u + 1]]:
            assert e[ids[u]] < s[ids[int(v)]], (u, int(v))
    g.close()


def test_stream_fanout_relays(S):
    g = S.Graph()
    hx = g.register(0x7f0000000000, 8, 8, 8)
    g.stream_begin(max_tasks=1024, max_tiles=4, max_records=1024, max_preds=4096)
    w0 = g.insert(S.OP_NOP, [hx], [S.WRITE])
    readers = [g.insert(S.OP_NOP, [hx], [S.READ]) for _ in range(300)]
    w1 = g.insert(S.OP_NOP, [hx], [S.WRITE])
    g.stream_end()
    rc, _ = g.wait()
    assert rc == 0
    ntasks = g.sizes()[0]
    assert ntasks > 302  # relays were appended (300 successors, 64 slots per task)
    s, e = g.tickets()
    for r in readers:
        assert e[w0] < s[r] and e[r] < s[w1]
    assert (e[:ntasks] > 0).all()
    g.close()


def test_stream_errors(S):
    g = S.Graph()
    hx = g.register(0x7f0000000000, 8, 8, 8)
    g.stream_begin(max_tasks=4, max_tiles=2, max_records=8, max_preds=16)
    for _ in range(4):
        g.insert(S.OP_NOP, [hx], [S.WRITE])
    with pytest.raises(S.SpxError) as ex:
        g.insert(S.OP_NOP, [hx], [S.WRITE])
    assert ex.value.code == S.ERR_QUEUE_FULL
    g.stream_end()
    rc, _ = g.wait()
    assert rc == 0
    with pytest.raises(S.SpxError) as ex:
        g.stream_flush()
    assert ex.value.code == S.ERR_STATE
    with pytest.raises(S.SpxError) as ex:
        g.insert(S.OP_NOP, [hx], [S.WRITE])
    assert ex.value.code == S.ERR_STATE
    g.close()
    g2 = S.Graph()  # an empty stream
    g2.stream_begin(max_tasks=8, max_tiles=2, max_records=8, max_preds=8)
    g2.stream_end()
    assert g2.wait()[0] == 0
    g2.close()


def test_stream_split_cholesky_bit_identical(S):
    """The split path streamed panel by panel (tiles with split slots, the
    kernel family fixed by the first panel inserted before the begin) gives
    the one-shot split graph's factor bit for bit."""
    from paper_2308_15964_b300 import cholesky
    n, b = 1536, 256
    T = n // b
    A = inputs.spd_matrix(n, 1.0, seed=5).numpy()
    Aref = torch.from_numpy(A.copy()).cuda()
    g0 = S.Graph()
    cholesky.cholesky_ozaki_graph(g0, Aref, b)
    assert g0.run()[0] == 0
    torch.cuda.synchronize()
    Lref = np.tril(Aref.cpu().numpy())
    g0.close()
    Ad = torch.from_numpy(A.copy()).cuda()
    store = cholesky.ozaki_store(n, b)
    slot = S.lib.spx_ozaki_slot_bytes(b)
    g = S.Graph()
    g.register_ozaki(store.data_ptr(), T * (T - 1) // 2, b)
    h = [[None] * T for _ in range(T)]
    for i in range(T):
        for j in range(i + 1):
            lo = store.data_ptr() + (i * (i - 1) // 2 + j) * slot if i > j else 0
            h[i][j] = g.register(Ad[i * b:, j * b:].data_ptr(), b, b, n, S.DT_F64, lo, b if lo else 0)
    R, W, OZ = S.READ, S.WRITE, S.F64_OZAKI

    def panel(k):
        t = g.insert(S.OP_POTRF, [h[k][k]], [W], 2)
        g.set_arg(t, k * b)
        for i in range(k + 1, T):
            g.insert(S.OP_TRSM, [h[k][k], h[i][k]], [R, W], 2 if i == k + 1 else 1, OZ)
        for i in range(k + 1, T):
            g.insert(S.OP_SYRK, [h[i][k], h[i][i]], [R, W], 2 if i == k + 1 else 1, OZ)
        for j in range(k + 1, T):
            for i in range(j + 1, T):
                g.insert(S.OP_GEMM_NT_SUB, [h[i][k], h[j][k], h[i][j]], [R, R, W],
                         (2 if i == k + 2 else 1) if j == k + 1 else 0, OZ)

    panel(0)
    g.stream_begin(max_tasks=512, max_tiles=T * T, max_records=2048, max_preds=4096)
    for k in range(1, T):
        panel(k)
        g.stream_flush()
    g.stream_end()
    rc, info = g.wait()
    assert rc == 0 and info == 0
    torch.cuda.synchronize()
    assert np.array_equal(np.tril(Ad.cpu().numpy()), Lref)
    g.close()


# --- end to end from host memory (spx_cholesky_host_ozaki) ------------------

@pytest.mark.parametrize("n,b", [(2000, 256), (1536, 128), (512, 512), (1100, 512)])
def test_host_entry_bit_identical(S, n, b):
    """The host-buffer entry (column blocks uploaded while the kernel runs)
    gives the same factor, bit for bit, as the device-resident split graph,
    and writes nothing above the diagonal blocks of L_host."""
    import torch
    from paper_2308_15964_b300 import cholesky, inputs
    A0 = inputs.spd_matrix(n, 0.1, seed=n + b)
    Ah = A0.clone().pin_memory()
    Lh = torch.full((n, n), 7.0, dtype=torch.float64).pin_memory()
    g = S.Graph()
    rc, info = cholesky.cholesky_host_ozaki(g, Ah, Lh, b)
    g.close()
    assert rc == 0 and info == 0
    Ad = A0.cuda()
    V = torch.zeros((n, min(b, n)), dtype=torch.float64, device="cuda")
    g = S.Graph()
    cholesky.cholesky_ozaki_graph(g, Ad, b, V=V)
    assert g.run()[0] == 0
    torch.cuda.synchronize()
    g.close()
    L = Lh.numpy()
    want = Ad.cpu().numpy()
    assert np.array_equal(np.tril(L), np.tril(want))
    # above the diagonal blocks: untouched
    T = -(-n // b)
    for j in range(1, T):
        assert (L[:j * b, j * b:(j + 1) * b] == 7.0).all()
    assert torch.equal(Ah, A0.pin_memory())  # the input is only read


def test_host_entry_not_spd(S):
    import torch
    from paper_2308_15964_b300 import cholesky, inputs
    n, b = 1024, 256
    A0 = inputs.spd_matrix(n, 1.0, seed=3)
    A0[700, 700] = -5.0
    Ah = A0.clone().pin_memory()
    Lh = torch.zeros((n, n), dtype=torch.float64).pin_memory()
    g = S.Graph()
    rc, info = cholesky.cholesky_host_ozaki(g, Ah, Lh, b)
    g.close()
    assert rc == S.NOT_SPD and info == 701


def test_tasks_done_while_streaming(S):
    """spx_graph_tasks_done: every task of a finished stream reads as done;
    tasks published behind a held chain read as not done while it runs."""
    import torch
    g = S.Graph()
    X = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    h = g.register_tensor(X)
    t0 = g.insert(S.OP_SPIN, [h], [S.WRITE])
    g.set_arg(t0, 300_000_000)
    g.stream_begin(max_tasks=64, max_tiles=4, max_records=64, max_preds=64)
    ids = [g.insert(S.OP_NOP, [h], [S.WRITE]) for _ in range(5)]
    g.stream_flush()
    early = g.tasks_done([t0] + ids)
    g.stream_end()
    assert g.wait()[0] == 0
    assert not early[1:].any()                   # behind the 0.3 s spin
    assert g.tasks_done([t0] + ids).all()
    start, end = g.tickets()
    assert (end < 2 ** 31).all()                 # the ticket alone
    g.close()
