"""GPU test of the serving loop: a short Poisson stream of FP64 and
TF32+refinement Cholesky-solve requests through the resident server, with
HBM-budget admission.  Every request completes; each result is bit-identical
to the same request run alone, and meets the FP64 backward-error bound
(TF32 requests after their refinement sweeps)."""
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


@pytest.mark.parametrize("split", [False, True])
def test_stream_alone_equals_mix(S, split):
    """split: FP64 requests of order >= 512 by split products in the
    one-CTA-per-SM server kernel (FP64 results)."""
    from paper_2308_15964_b300 import serve
    nmax, rhs_max, seed = 1536, 8, 3
    if split:
        serve.SPLIT_MIN_N, keep_min = 512, serve.SPLIT_MIN_N
    try:
        out, finished, arena = serve.serve(rate=30, duration=1.0, budget=4e9, seed=seed,
                                           nmax=nmax, rhs_max=rhs_max, keep_results=True,
                                           max_wall=300, split_fp64=split)
    finally:
        if split:
            serve.SPLIT_MIN_N = keep_min
    assert out["completed"] == out["requests"] > 5 and out["failed"] == 0
    assert out["tf32_requests"] >= 1
    assert (out["split_fp64_requests"] >= 1) == split
    A_all = inputs.spd_matrix(nmax, 1.0, seed)
    B_all = inputs.rhs(nmax, rhs_max, seed)
    src = serve.Sources(nmax, rhs_max, seed)
    alone_arena = serve.Arena(int(1.5e9))
    stream = torch.cuda.Stream()
    for q in finished:
        n, r = q.n, q.nrhs
        A = A_all[:n, :n].numpy().copy()
        B = B_all[:n, :r].numpy().copy()
        X = q.views["X"].cpu().numpy()
        assert O.solve_backward_error(A, X, B).max() <= 1e-14, (q.n, q.prec)
        # alone: same request on fresh buffers through a private graph
        q2 = serve.Request(q.idx, 0.0, n, r, q.prec, q.tile, split=q.split)
        q2.bytes = serve.request_bytes(n, r, q.prec, q.split)
        q2.offset = alone_arena.alloc(q2.bytes)
        assert q2.offset >= 0
        g = serve.build_graph(q2, alone_arena, src, stream)
        rc, _ = g.run()
        g.close()
        assert rc == 0
        assert torch.equal(q2.views["X"], q.views["X"])
        assert torch.equal(q2.views["A"], q.views["A"])
        alone_arena.release(q2.offset, q2.bytes)
