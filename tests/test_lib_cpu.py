"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports
every symbol the headers declare, and validates arguments on the host
(no device call is made here)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    from paper_2308_15964_b300 import build
    build.build()
    from paper_2308_15964_b300 import spx
    return spx


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(spx_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_exports_every_declared_symbol(S):
    names = declared_functions()
    assert len(names) >= 20
    lib = ctypes.CDLL(S.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert S.lib.spx_abi_version() == 1


def test_strerror(S):
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8, -9):
        assert S.strerror(code) and S.strerror(code) != "unknown status code"
    assert S.strerror(-99) == "unknown status code"


FAKE = 0x7f0000000000   # host-side validation never dereferences tile pointers


def fake_tiles(g, n, b):
    T = n // b
    h = {}
    for i in range(T):
        for j in range(T):
            h[i, j] = g.register(FAKE + 8 * (i * b * n + j * b), b, b, n)
    return h


def test_register_validation(S):
    g = S.Graph()
    with pytest.raises(S.SpxError) as e:
        g.register(0, 4, 4, 4)
    assert e.value.code == S.ERR_INVALID_ARG
    for bad in [(FAKE, 0, 4, 4), (FAKE, 4, 0, 4), (FAKE, 4, 8, 4)]:
        with pytest.raises(S.SpxError):
            g.register(*bad)
    h1 = g.register(FAKE, 4, 4, 8)
    assert g.register(FAKE, 4, 4, 8) == h1          # same address, same handle
    with pytest.raises(S.SpxError):
        g.register(FAKE, 4, 5, 8)                    # same address, other shape
    h2 = g.register(FAKE + 32, 4, 4, 8)
    assert h2 == h1 + 1
    g.close()


def test_insert_validation(S):
    g = S.Graph()
    h = fake_tiles(g, 256, 64)
    R, W, C = S.READ, S.WRITE, S.COMMUTATIVE_WRITE
    assert g.insert(S.OP_POTRF, [h[0, 0]], [W]) == 0
    assert g.insert(S.OP_TRSM, [h[0, 0], h[1, 0]], [R, W]) == 1
    assert g.insert(S.OP_GEMM_NT_SUB, [h[1, 0], h[2, 0], h[2, 1]], [R, R, C]) == 2
    bad = [
        (S.OP_POTRF, [h[0, 0]], [R]),                       # written operand read-only
        (S.OP_TRSM, [h[0, 0]], [R]),                        # operand count
        (S.OP_GEMM_NT_SUB, [h[1, 0], h[1, 0], h[1, 1]], [R, R, W]),  # repeated operand
        (99, [h[0, 0]], [W]),                               # unknown op
        (S.OP_NOP, [h[0, 0]], [7]),                         # unknown mode
    ]
    for op, hh, mm in bad:
        with pytest.raises(S.SpxError) as e:
            g.insert(op, hh, mm)
        assert e.value.code == S.ERR_INVALID_ARG
    with pytest.raises(S.SpxError) as e:
        g.insert(S.OP_NOP, [12345], [R])
    assert e.value.code == S.ERR_BAD_HANDLE
    with pytest.raises(S.SpxError):
        g.insert(S.OP_NOP, [h[0, 0]], [R], prec=9)
    # shape mismatch: TRSM needs A_ik.cols == L_kk.rows
    odd = g.register(FAKE + (1 << 30), 64, 32, 64)
    with pytest.raises(S.SpxError):
        g.insert(S.OP_TRSM, [h[0, 0], odd], [R, W])
    # NOP / SPIN accept any handles and modes, repeated handles merge
    assert g.insert(S.OP_NOP, [h[0, 0], h[0, 0], h[1, 1]], [R, C, W]) == 3
    with pytest.raises(S.SpxError) as e:
        g.set_arg(100, 5)
    assert e.value.code == S.ERR_BAD_HANDLE
    g.set_arg(0, 64)
    n, ne, nacc, nt = g.sizes()
    assert (n, nacc, nt) == (4, 1 + 2 + 3 + 2, 17) and ne == -1
    g.close()


def test_state_errors(S):
    g = S.Graph()
    rc, info = g.wait()
    assert rc == S.ERR_STATE
    with pytest.raises(S.SpxError) as e:
        g.edges()
    assert e.value.code == S.ERR_STATE
    with pytest.raises(S.SpxError):
        g.reset()
    with pytest.raises(S.SpxError) as e:
        g.execute(0)                                    # empty graph
    assert e.value.code == S.ERR_STATE
    h = g.register(FAKE, 8, 8, 8)
    g.insert(S.OP_NOP, [h], [S.WRITE])
    g.clear()
    assert g.sizes()[0] == 0 and g.sizes()[3] == 0
    g.close()
    g.close()


def test_config_validation(S):
    with pytest.raises(S.SpxError):
        S.Graph(executor=7)
    with pytest.raises(S.SpxError):
        S.Graph(num_ctas=-1)


def test_batch_validation(S):
    """spx_batch_execute refuses bad batches on the host, before any device
    work: no graphs, a graph given twice, an empty graph, and one tile
    address registered with two shapes in two members."""
    import ctypes
    assert S.lib.spx_batch_execute(None, 1, None) == S.ERR_INVALID_ARG
    g1, g2, g3 = S.Graph(), S.Graph(), S.Graph()
    h1 = g1.register(FAKE, 8, 8, 8)
    g1.insert(S.OP_NOP, [h1], [S.WRITE])
    h2 = g2.register(FAKE, 8, 4, 8)                 # same address, other shape
    g2.insert(S.OP_NOP, [h2], [S.WRITE])
    arr = (ctypes.c_void_p * 2)(g1._h.value, g1._h.value)
    assert S.lib.spx_batch_execute(arr, 0, None) == S.ERR_INVALID_ARG
    assert S.lib.spx_batch_execute(arr, 2, None) == S.ERR_INVALID_ARG   # g1 twice
    with pytest.raises(S.SpxError) as e:
        S.batch_execute([g1, g3], 0)                # g3 has no task
    assert e.value.code == S.ERR_STATE
    with pytest.raises(S.SpxError) as e:
        S.batch_execute([g1, g2], 0)                # tile shape conflict
    assert e.value.code == S.ERR_INVALID_ARG
    assert g1.wait()[0] == S.ERR_STATE              # nothing started
    for g in (g1, g2, g3):
        g.close()


@pytest.mark.parametrize("seed", range(12))
def test_bottom_level_priorities_match_oracle_dag(S, seed):
    """spx_graph_assign_priorities computes top and bottom levels from the
    access records alone; the classes must equal those from longest paths on
    the DAG the oracle derives (unit weights: NOP tasks have one phase):
    slack 0 -> 2, slack <= CP/10 -> 1, else 0."""
    from oracle import oracle as O
    from paper_2308_15964_b300 import inputs
    n = [5, 40, 120, 300][seed % 4]
    t, k, m = inputs.random_access_lists(n, 1 + seed % 7, 4, seed=4242 + seed, nmodes=5)
    ntask = int(t.max()) + 1
    g = S.Graph()
    handles = {}
    for key in np.unique(k):
        handles[int(key)] = g.register(FAKE + 4096 * int(key), 8, 8, 8)
    i = 0
    while i < len(t):
        j = i
        while j < len(t) and t[j] == t[i]:
            j += 1
        g.insert(S.OP_NOP, [handles[int(x)] for x in k[i:j]], [int(x) for x in m[i:j]])
        i = j
    g.assign_priorities()
    _, got = g.task_ops()
    rp, col, _ = O.derive(ntask, t, k, m)
    tl = np.zeros(ntask)
    for u in range(ntask):
        for p in range(rp[u], rp[u + 1]):
            v = int(col[p])
            tl[v] = max(tl[v], tl[u] + 1)
    bl = np.ones(ntask)
    for u in range(ntask - 1, -1, -1):
        for p in range(rp[u], rp[u + 1]):
            bl[u] = max(bl[u], 1 + bl[int(col[p])])
    cp = (tl + bl).max()
    slack = cp - tl - bl
    want = np.where(slack <= 1e-9 * cp, 2, np.where(slack <= 0.1 * cp, 1, 0))
    assert np.array_equal(got, want), (got, want)
    g.close()


def test_streaming_and_host_entry_validation(S):
    """The streaming upload, the completion query and the host-memory
    Cholesky refuse bad use on the host, before any device call."""
    g = S.Graph()
    h = g.register(FAKE, 8, 8, 8)
    g.insert(S.OP_NOP, [h], [S.WRITE])
    buf = (ctypes.c_double * 64)()
    # not streaming: no upload
    rc = S.lib.spx_stream_copy_h2d(g._h, ctypes.c_void_p(FAKE), 64, buf, 64, 64, 8)
    assert rc == S.ERR_STATE
    # width above a pitch
    rc = S.lib.spx_stream_copy_h2d(g._h, ctypes.c_void_p(FAKE), 32, buf, 64, 64, 8)
    assert rc == S.ERR_INVALID_ARG
    # not launched: no completion snapshot
    t = np.zeros(1, dtype=np.uint32)
    d = np.zeros(1, dtype=np.int32)
    rc = S.lib.spx_graph_tasks_done(g._h, t.ctypes.data_as(ctypes.c_void_p), 1,
                                    d.ctypes.data_as(ctypes.c_void_p))
    assert rc == S.ERR_STATE
    rc = S.lib.spx_graph_tasks_done(g._h, None, -1, None)
    assert rc == S.ERR_INVALID_ARG
    g.close()
    g = S.Graph()
    info = ctypes.c_int(7)
    # null host buffers, a tile that is no multiple of 32, a short leading dimension
    for args in ((None, buf, 64, 64, 64, FAKE, 64), (buf, buf, 64, 64, 48, FAKE, 64),
                 (buf, buf, 64, 32, 64, FAKE, 64)):
        ha, hl, n, ldh, b, dA, lda = args
        rc = S.lib.spx_cholesky_host_ozaki(g._h, ha, hl, n, ldh, b, ctypes.c_void_p(dA), lda,
                                           ctypes.c_void_p(FAKE), 1 << 20, ctypes.c_void_p(FAKE),
                                           64, None, ctypes.byref(info))
        assert rc == S.ERR_INVALID_ARG and info.value == 0
    g.close()


@pytest.mark.parametrize("n,b", [(1024, 256), (1000, 256), (512, 512), (96, 32)])
@pytest.mark.parametrize("inverse_panels", [False, True])
def test_split_store_size_is_what_the_library_requires(S, n, b, inverse_panels):
    """cholesky.ozaki_store's size passes the library's host-side check, one
    slot less does not (the exact size gets as far as the first CUDA call,
    which has no device here); one tile without inverse panels needs none."""
    from paper_2308_15964_b300 import cholesky
    store = cholesky.ozaki_store(n, b, device="cpu", inverse_panels=inverse_panels)
    slot = S.lib.spx_ozaki_slot_bytes(b)
    T = -(-n // b)
    need = T * (T - 1) // 2 + (T if inverse_panels else 0)
    assert store.numel() == max(1, need) * slot
    cases = [(store.numel(), True)] + ([(store.numel() - slot, False)] if need else [])
    for nbytes, want_ok in cases:
        g = S.Graph()
        nt = ctypes.c_longlong()
        rc = S.lib.spx_cholesky_insert_ozaki(
            g._h, ctypes.c_void_p(FAKE), n, n, b, ctypes.c_void_p(FAKE + (1 << 32)),
            ctypes.c_longlong(nbytes), ctypes.c_void_p(FAKE + (1 << 33)) if inverse_panels else None,
            b if inverse_panels else 0, 0, None, 0, 0, 1, ctypes.byref(nt))
        g.close()
        if want_ok:
            assert rc in (S.OK, S.ERR_CUDA), rc
        else:
            assert rc == S.ERR_INVALID_ARG, rc
