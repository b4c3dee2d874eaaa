"""The allocation-free derivation entry point against the oracle.

spx_graph_derive_noalloc serves callers that cannot allocate device memory
(host callbacks, runtimes that own every device byte through their own
pool, servers that must not touch the allocator while serving): they hold
the access records in their own device buffers and get the successor CSR
back without the library calling cudaMalloc.  Here the test allocates those
buffers (it is the caller) and checks, on two calls in a row, that the
result is bit-identical to the CPU oracle's derivation of the same access
lists (the tolerance of every DAG test: exact), and that the graph path
(spx_graph_derive) agrees too.  Malformed records, a too-small output and
an edge count beyond 2^32 are refused before anything is written.  This file
is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2308_15964_b300 import inputs
from tests._gpu import need_cuda, nop_graph, spx_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    need_cuda()
    return spx_mod()


def records(t, k, m, nkeys):
    """Per-task records sorted by handle, with each handle's list position."""
    n = int(t.max()) + 1
    task_rec = [0]
    rh, rs, rm = [], [], []
    count = np.zeros(nkeys, np.int64)
    i = 0
    for u in range(n):
        j = i
        while j < len(t) and t[j] == u:
            j += 1
        for kk, mm in sorted(zip(k[i:j].tolist(), m[i:j].tolist())):
            rh.append(kk)
            rm.append(mm)
            rs.append(int(count[kk]))
            count[kk] += 1
        task_rec.append(len(rh))
        i = j
    return n, (np.asarray(task_rec, np.uint32), np.asarray(rh, np.uint32),
               np.asarray(rs, np.uint32), np.asarray(rm, np.uint8))


def call_noalloc(S, n, nkeys, rec, col_cap, col_fill=0):
    task_rec, rh, rs, rm = (torch.from_numpy(x).cuda() for x in rec)
    row_ptr = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    col = torch.full((max(col_cap, 1),), col_fill, dtype=torch.int32, device="cuda")
    indeg = torch.full((n,), col_fill, dtype=torch.int32, device="cuda")
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    P = ctypes.c_void_p
    rc = S.lib.spx_graph_derive_noalloc(
        P(task_rec.data_ptr()), P(rh.data_ptr()), P(rs.data_ptr()), P(rm.data_ptr()), n, nkeys,
        len(rh), P(row_ptr.data_ptr()), P(col.data_ptr()), col_cap, P(indeg.data_ptr()),
        P(status.data_ptr()), P(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    u32 = lambda x: x.cpu().numpy().view(np.uint32)
    return int(status.item()), u32(row_ptr), u32(col), u32(indeg)


def graph_path(S, t, k, m):
    n = int(t.max()) + 1
    g = nop_graph(S, n, t, k, m)
    g.derive()
    out = g.edges()
    g.close()
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_oracle_twice(S, seed):
    cases = []
    for j, (ntask, nkeys) in enumerate(((300, 12), (2000, 64))):
        t, k, m = inputs.random_access_lists(ntask, nkeys, 5, seed=9000 + 10 * seed + j,
                                             allow_repeats=False)
        n, rec = records(t, k, m, nkeys)
        cases.append((t, k, m, n, nkeys, rec))
    # two calls in a row, different graphs, then the first again: the shared
    # scratch must not carry anything from one call into the next
    for t, k, m, n, nkeys, rec in cases + cases[:1]:
        rp, col, deg = O.derive(n, t, k, m)
        st, rp2, col2, deg2 = call_noalloc(S, n, nkeys, rec, col_cap=4 * len(rec[1]) + 16)
        assert st == 0
        assert np.array_equal(rp2, rp)
        assert np.array_equal(col2[:len(col)], col)
        assert np.array_equal(deg2, deg)
    # the graph path gives the same CSR
    t, k, m, n, nkeys, rec = cases[0]
    rpg, colg, degg = graph_path(S, t, k, m)
    rp, col, deg = O.derive(n, t, k, m)
    assert np.array_equal(rpg, rp) and np.array_equal(colg, col) and np.array_equal(degg, deg)


def test_rejections(S):
    t, k, m = inputs.random_access_lists(100, 8, 4, seed=4, allow_repeats=False)
    n, rec = records(t, k, m, 8)
    rp, col, deg = O.derive(n, t, k, m)
    # output too small: status set, row_ptr[n] holds the edge count, col and
    # indeg untouched
    st, rp2, col2, deg2 = call_noalloc(S, n, 8, rec, col_cap=max(0, len(col) - 1), col_fill=-7)
    assert st == S.ERR_INVALID_ARG and rp2[n] == len(col)
    assert (col2 == np.uint32(2 ** 32 - 7)).all() and (deg2 == np.uint32(2 ** 32 - 7)).all()
    # malformed: a list position out of range, and a handle past nhandles
    bad = list(rec)
    bad[2] = rec[2].copy()
    bad[2][0] = 999
    st, _, _, _ = call_noalloc(S, n, 8, tuple(bad), col_cap=4 * len(rec[1]))
    assert st == S.ERR_INVALID_ARG
    bad = list(rec)
    bad[1] = rec[1].copy()
    bad[1][3] = 8
    st, _, _, _ = call_noalloc(S, n, 8, tuple(bad), col_cap=4 * len(rec[1]))
    assert st == S.ERR_INVALID_ARG
    # malformed: one task names the same handle twice (positions 0 and 1 of
    # handle 0 both belong to task 0)
    dup = (np.array([0, 2, 3], np.uint32), np.array([0, 0, 0], np.uint32),
           np.array([0, 1, 2], np.uint32), np.array([1, 1, 1], np.uint8))
    st, _, _, _ = call_noalloc(S, 2, 1, dup, col_cap=16)
    assert st == S.ERR_INVALID_ARG
    # and a good call right after the failed ones
    st, rp3, col3, deg3 = call_noalloc(S, n, 8, rec, col_cap=4 * len(rec[1]))
    assert st == 0 and np.array_equal(rp3, rp) and np.array_equal(col3[:len(col)], col)
    assert np.array_equal(deg3, deg)
    # sizes beyond the fixed scratch are refused on the host, before any launch
    P = ctypes.c_void_p
    one = P(1)
    assert S.lib.spx_graph_derive_noalloc(one, one, one, one, 4, 4, (1 << 18) + 1, one, one, 10,
                                          one, one, None) == S.ERR_INVALID_ARG
    assert S.lib.spx_graph_derive_noalloc(one, one, one, one, 4, (1 << 16) + 1, 8, one, one, 10,
                                          one, one, None) == S.ERR_INVALID_ARG


def test_edge_count_beyond_32_bits(S):
    """65536 READs followed by 65536 COMMUTATIVE_WRITEs on one handle: every
    write depends on every read, 2^32 edges (a valid list within the record
    limit).  The total does not fit the 32-bit output: refused with
    row_ptr[n] saturated, nothing written to col or indeg."""
    R = C = 1 << 16
    n = R + C
    task_rec = np.arange(n + 1, dtype=np.uint32)
    rh = np.zeros(n, np.uint32)
    rs = np.arange(n, dtype=np.uint32)
    rm = np.concatenate([np.zeros(R, np.uint8), np.full(C, 2, np.uint8)])
    st, rp, col, deg = call_noalloc(S, n, 1, (task_rec, rh, rs, rm), col_cap=1024, col_fill=-3)
    assert st == S.ERR_INVALID_ARG
    assert rp[n] == 0xFFFFFFFF
    assert (col == np.uint32(2 ** 32 - 3)).all() and (deg == np.uint32(2 ** 32 - 3)).all()
    # the same shape one size smaller fits 32 bits: E = R C exactly
    R2 = C2 = 1 << 10
    n2 = R2 + C2
    rec2 = (np.arange(n2 + 1, dtype=np.uint32), np.zeros(n2, np.uint32),
            np.arange(n2, dtype=np.uint32),
            np.concatenate([np.zeros(R2, np.uint8), np.full(C2, 2, np.uint8)]))
    st, rp, col, deg = call_noalloc(S, n2, 1, rec2, col_cap=R2 * C2)
    assert st == 0 and rp[n2] == R2 * C2
    t = np.arange(n2, dtype=np.uint32)
    orp, ocol, odeg = O.derive(n2, t, np.zeros(n2, np.uint64), rec2[3].astype(np.int32))
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol) and np.array_equal(deg, odeg)
