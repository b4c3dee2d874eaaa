"""The split-FP64 path in the resident server (tensor_cores = 2: the
one-CTA-per-SM kernel that owns all of TMEM).  The TF32 / BF16 tensor-core
ops run unchanged in that kernel (a mixed factorization there is bit-identical
to the two-CTA-per-SM run); split-FP64, TF32 and FP64 requests submitted while
the others run each equal the same graph run alone, bit for bit, and the
split request's factor and solution meet the FP64 tolerances against the
oracle; servers without that kernel refuse split requests."""
import time

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2308_15964_b300 import inputs
from tests._gpu import need_cuda, spx_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    need_cuda()
    return spx_mod()


def force_split_kernel(S, g, keep):
    """Add a SPLIT task on a tile of its own, so that the graph runs in the
    one-CTA-per-SM kernel; the task touches nothing else."""
    b = 64
    slot = S.lib.spx_ozaki_slot_bytes(b)
    store = torch.zeros(slot, dtype=torch.uint8, device="cuda")
    Z = torch.ones((b, b), dtype=torch.float64, device="cuda")
    keep += [store, Z]
    g.register_ozaki(store.data_ptr(), 1, b)
    h = g.register(Z.data_ptr(), b, b, b, S.DT_F64, store.data_ptr(), b)
    g.insert(S.OP_SPLIT, [h], [S.WRITE], prec=S.F64_OZAKI)


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tensor_core_ops_in_split_kernel(S, prec):
    from paper_2308_15964_b300 import mixed
    p = S.TF32 if prec == "tf32" else S.BF16
    n, b = 1280, 256
    A = inputs.spd_matrix(n, 0.01, seed=21, device="cuda")
    X = inputs.rhs(n, 3, seed=21, device="cuda")
    outs = []
    for split_kernel in (False, True):
        Ad, Xd = A.clone(), X.clone()
        Alo = torch.zeros((n, n), dtype=mixed.lowp_dtype(p), device="cuda")
        V = torch.zeros((n, b), dtype=torch.float64, device="cuda")
        g = S.Graph()
        keep = []
        mixed.factor_graph(g, Ad, Alo, b, Xd, p, V=V)
        if split_kernel:
            force_split_kernel(S, g, keep)
        rc, info = g.run()
        torch.cuda.synchronize()
        assert rc == 0 and info == 0
        g.close()
        outs.append((Ad, Xd))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def wait_all(srv, ids, timeout=120.0):
    done = {}
    t0 = time.time()
    while len(done) < len(ids):
        for r in ids:
            if r not in done:
                res = srv.poll(r)
                if res is not None:
                    done[r] = res
        assert time.time() - t0 < timeout
    return done


def build(S, kind, n, b, nrhs, seed):
    """(graph, tensors to check, keep-alive list) of one request."""
    from paper_2308_15964_b300 import cholesky, mixed
    A = inputs.spd_matrix(n, 1.0, seed, device="cuda")
    X = inputs.rhs(n, nrhs, seed, device="cuda")
    g = S.Graph()
    keep = [A, X]
    if kind == "split":
        V = torch.zeros((n, b), dtype=torch.float64, device="cuda")
        keep.append(V)
        cholesky.cholesky_ozaki_graph(g, A, b, X, V=V)
    elif kind == "tf32":
        Alo = torch.zeros((n, n), dtype=torch.float32, device="cuda")
        V = torch.zeros((n, b), dtype=torch.float64, device="cuda")
        keep += [Alo, V]
        mixed.factor_graph(g, A, Alo, b, X, S.TF32, V=V)
    else:
        cholesky.cholesky_graph(g, A, b, X)
    # the inputs are made by kernels on torch's stream; the resident kernel
    # may start a submitted request at once
    torch.cuda.synchronize()
    return g, (A, X), keep


def test_split_requests_in_server(S):
    specs = [("split", 1536, 256, 2, 31), ("tf32", 1024, 256, 3, 32), ("f64", 777, 128, 1, 33),
             ("split", 2048, 512, 4, 34), ("split", 640, 128, 1, 35), ("f64", 1000, 256, 2, 36)]
    srv = S.Server(tensor_cores=2, idle_ns=500_000_000)
    reqs = []
    for kind, n, b, r, seed in specs:       # submitted while the earlier ones run
        g, outs, keep = build(S, kind, n, b, r, seed)
        rid = srv.submit(g)
        assert rid is not None
        g.close()
        reqs.append((kind, n, b, r, seed, rid, outs, keep))
    done = wait_all(srv, [q[5] for q in reqs])
    assert all(done[q[5]] == (0, 0) for q in reqs), [(q[0], q[1], done[q[5]]) for q in reqs]
    assert srv.stop() == 0
    srv.close()
    for kind, n, b, r, seed, rid, (A, X), _ in reqs:
        g, (A1, X1), keep = build(S, kind, n, b, r, seed)
        rc, info = g.run()
        torch.cuda.synchronize()
        g.close()
        assert rc == 0 and info == 0
        assert torch.equal(A, A1) and torch.equal(X, X1), (kind, n)
        if kind == "split":  # FP64 tolerances against the oracle
            A0 = inputs.spd_matrix(n, 1.0, seed).numpy()
            B0 = inputs.rhs(n, r, seed).numpy()
            Lo, Xo = A0.copy(), B0.copy()
            assert O.tiled_cholesky(Lo, b, Xo) == 0
            L = np.tril(A.cpu().numpy())
            assert np.abs(L - np.tril(Lo)).max() / np.abs(np.tril(Lo)).max() <= 1e-12
            assert O.solve_backward_error(A0, X.cpu().numpy(), B0).max() <= 1e-14


def test_split_request_refused_without_split_kernel(S):
    g, _, keep = build(S, "split", 512, 128, 1, 40)
    for tc in (0, 1):
        srv = S.Server(tensor_cores=tc, idle_ns=100_000_000)
        with pytest.raises(S.SpxError):
            srv.submit(g)
        srv.close()
    g.close()
    with pytest.raises(S.SpxError):
        S.Server(tensor_cores=3)
