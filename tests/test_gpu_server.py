"""GPU tests of the continuous-batching server: requests submitted while
others run are admitted, derived on the device and interleaved in one
resident persistent kernel; each result equals the same request run alone
(bit for bit: the same tile code runs the same units) and the oracle's
(FP64 tolerances); a failing request reports its own status without
disturbing the others; the resident kernel exits when idle and is
relaunched by the next submission."""
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


def make_request(S, n, b, nrhs, seed, bad_col=None):
    from paper_2308_15964_b300 import cholesky
    A = inputs.spd_matrix(n, 1.0, seed)
    if bad_col is not None:
        A[bad_col - 1, bad_col - 1] = -1.0
    B = inputs.rhs(n, nrhs, seed)
    Ad, Bd = A.cuda(), B.cuda()
    g = S.Graph()
    cholesky.cholesky_graph(g, Ad, b, Bd)
    return {"A": A, "B": B, "Ad": Ad, "Bd": Bd, "g": g, "n": n, "b": b}


def wait_all(srv, ids, timeout=60.0):
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


def run_alone(S, req):
    from paper_2308_15964_b300 import cholesky
    Ad, Bd = req["A"].cuda(), req["B"].cuda()
    g = S.Graph()
    cholesky.cholesky_graph(g, Ad, req["b"], Bd)
    rc, info = g.run()
    g.close()
    return rc, info, Ad, Bd


def test_mixed_requests_alone_equals_mix(S):
    srv = S.Server(idle_ns=500_000_000)
    sizes = [(96, 32, 1), (512, 64, 2), (1000, 128, 3), (64, 64, 1), (2048, 512, 1), (300, 64, 4),
             (777, 256, 2), (128, 32, 1)]
    reqs = [make_request(S, n, b, r, seed=100 + i) for i, (n, b, r) in enumerate(sizes)]
    ids = []
    for req in reqs:                       # submit while earlier ones run
        rid = srv.submit(req["g"])
        assert rid is not None
        req["g"].close()                   # the server keeps its own copy
        ids.append(rid)
    done = wait_all(srv, ids)
    assert all(done[r] == (0, 0) for r in ids)
    for req in reqs:
        rc, info, La, Xa = run_alone(S, req)
        assert rc == 0
        assert torch.equal(La, req["Ad"]) and torch.equal(Xa, req["Bd"])
        L = req["Ad"].cpu().numpy()
        Lo = req["A"].numpy().copy()
        Xo = req["B"].numpy().copy()
        assert O.tiled_cholesky(Lo, req["b"], Xo) == 0
        err = np.abs(np.tril(L) - np.tril(Lo)).max() / np.abs(np.tril(Lo)).max()
        assert err <= 1e-12
        assert O.solve_backward_error(req["A"].numpy(), req["Bd"].cpu().numpy(), req["B"].numpy()).max() <= 1e-14
    assert srv.stop() == 0
    st = srv.stats()
    assert st["requests"] == len(sizes) and st["live"] == 0
    srv.close()


def test_failing_request_isolated(S):
    srv = S.Server(idle_ns=500_000_000)
    good1 = make_request(S, 512, 64, 1, seed=7)
    bad = make_request(S, 400, 64, 1, seed=8, bad_col=130)
    good2 = make_request(S, 640, 128, 2, seed=9)
    ids = [srv.submit(r["g"]) for r in (good1, bad, good2)]
    done = wait_all(srv, ids)
    expect = O.tiled_cholesky(bad["A"].numpy().copy(), 64)
    assert done[ids[1]] == (S.NOT_SPD, expect)
    assert done[ids[0]] == (0, 0) and done[ids[2]] == (0, 0)
    for r in (good1, good2):
        rc, _, La, Xa = run_alone(S, r)
        assert torch.equal(La, r["Ad"]) and torch.equal(Xa, r["Bd"])
    assert srv.stop() == 0
    srv.close()


def test_idle_exit_and_relaunch(S):
    srv = S.Server(idle_ns=50_000_000)
    r1 = make_request(S, 256, 64, 1, seed=11)
    i1 = srv.submit(r1["g"])
    wait_all(srv, [i1])
    time.sleep(0.3)                        # resident kernel leaves after 50 ms idle
    r2 = make_request(S, 256, 64, 1, seed=12)
    i2 = srv.submit(r2["g"])
    assert wait_all(srv, [i2])[i2] == (0, 0)
    rc, _, La, _ = run_alone(S, r2)
    assert torch.equal(La, r2["Ad"])
    assert srv.stop() == 0
    srv.close()


def test_admission_when_full(S):
    # tiny pools: a second large request must wait for the first to finish
    srv = S.Server(max_tasks=300, max_tiles=200, max_records=1200, max_edges=1500,
                   idle_ns=500_000_000)
    a = make_request(S, 1024, 128, 1, seed=21)       # 120 + 72 tasks
    b = make_request(S, 1024, 128, 1, seed=22)
    ia = srv.submit(a["g"])
    assert ia is not None
    ib = srv.submit(b["g"])
    assert ib is None                                 # no room until a finishes
    wait_all(srv, [ia])
    ib = srv.submit(b["g"])
    assert ib is not None
    assert wait_all(srv, [ib])[ib] == (0, 0)
    assert srv.stop() == 0
    srv.close()
