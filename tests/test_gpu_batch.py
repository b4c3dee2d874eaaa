"""GPU parity of the batched path: many uneven Cholesky solves inserted into
one graph and run by one persistent launch, against the oracle problem by
problem; alone-vs-batch bit-identity; CUDA-graph replay; the autotuner."""
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


def check_problem(batch, i, b):
    A = inputs.spd_matrix(int(batch.n[i]), batch.sigma, batch.seed_of(i)).numpy()
    B = inputs.rhs(int(batch.n[i]), int(batch.nrhs[i]), batch.seed_of(i)).numpy()
    L = batch.a_view(i).cpu().numpy()
    X = batch.x_view(i).cpu().numpy()
    Lo, Xo = A.copy(), B.copy()
    assert O.tiled_cholesky(Lo, b, Xo) == 0
    err = np.abs(np.tril(L) - np.tril(Lo)).max() / np.abs(np.tril(Lo)).max()
    assert err <= 1e-12, (i, err)
    assert O.solve_backward_error(A, X, B).max() <= 1e-14


def test_batch_vs_oracle_and_alone(S):
    from paper_2308_15964_b300 import batch as Bt
    n, r = Bt.problem_sizes(96, seed=5, nmax=384)
    tiles = [[32, 64, 128, 256][i % 4] for i in range(len(n))]
    bt = Bt.Batch(n, r, seed=5)
    g = S.Graph(cuda_graph=True)
    ntask = Bt.insert(g, bt, tiles)
    assert ntask == g.sizes()[0]
    rc, _ = g.run()
    assert rc == 0
    for i in range(len(n)):
        check_problem(bt, i, tiles[i])
    first = (bt.A.clone(), bt.X.clone())
    # replay the same batch through the captured CUDA graph: bit-identical
    for _ in range(2):
        g.reset()
        bt.restore()
        rc, _ = g.run()
        assert rc == 0
        assert torch.equal(bt.A, first[0]) and torch.equal(bt.X, first[1])
    g.close()
    # a problem run alone gives the same bits as inside the batch
    for i in (0, 7, 50):
        one = Bt.Batch([n[i]], [r[i]], seed=5, fill=False)
        one.seed = bt.seed
        one.a_view(0).copy_(bt.A0[int(bt.a_off[i]):int(bt.a_off[i]) + int(n[i]) ** 2].view(int(n[i]), -1))
        one.x_view(0).copy_(bt.X0[int(bt.x_off[i]):int(bt.x_off[i]) + int(n[i] * r[i])].view(int(n[i]), -1))
        g1 = S.Graph()
        Bt.insert(g1, one, [tiles[i]])
        assert g1.run()[0] == 0
        assert torch.equal(one.a_view(0), bt.a_view(i)) and torch.equal(one.x_view(0), bt.x_view(i))
        g1.close()


def test_per_task_cuda_graph_replay(S):
    from paper_2308_15964_b300 import batch as Bt
    n, r = Bt.problem_sizes(12, seed=6, nmax=256)
    bt = Bt.Batch(n, r, seed=6)
    tiles = [64] * len(n)
    outs = []
    for ex in (S.EXEC_PERSISTENT, S.EXEC_PER_TASK, S.EXEC_STREAMS):
        g = S.Graph(executor=ex, cuda_graph=True)
        Bt.insert(g, bt, tiles)
        for rep in range(3):
            bt.restore()
            rc, _ = g.run()
            assert rc == 0
            g.reset()
        outs.append((bt.A.clone(), bt.X.clone()))
        g.close()
    for o in outs[1:]:
        assert torch.equal(outs[0][0], o[0]) and torch.equal(outs[0][1], o[1])


def test_autotune_small(S):
    from paper_2308_15964_b300 import batch as Bt
    best, table = Bt.autotune([96, 160], copies=8)
    assert set(best) == {96, 160}
    assert set(table[96]) == {32, 64, 128} and set(table[160]) == {32, 64, 128, 256}
    assert all(t > 0 for v in table.values() for t in v.values())


def test_split_batch_vs_oracle_and_alone(S):
    """The batch with every problem on the split path (trailing updates and
    inverse panel products split on the tensor cores): each problem within
    the FP64 tolerances of the oracle, bit-identical alone and in the batch,
    and on CUDA-graph replay; the autotuner in the same mode."""
    from paper_2308_15964_b300 import batch as Bt
    n, r = Bt.problem_sizes(48, seed=7, nmax=512)
    tiles = [[32, 64, 128, 256][i % 4] for i in range(len(n))]
    bt = Bt.Batch(n, r, seed=7)
    g = S.Graph(cuda_graph=True)
    ntask = Bt.insert(g, bt, tiles, split=True)
    assert ntask == g.sizes()[0]
    assert g.run()[0] == 0
    for i in range(len(n)):
        check_problem(bt, i, tiles[i])
    first = (bt.A.clone(), bt.X.clone())
    g.reset()
    bt.restore()
    assert g.run()[0] == 0
    assert torch.equal(bt.A, first[0]) and torch.equal(bt.X, first[1])
    g.close()
    for i in (0, 5, 31):
        one = Bt.Batch([n[i]], [r[i]], seed=7, fill=False)
        one.a_view(0).copy_(bt.A0[int(bt.a_off[i]):int(bt.a_off[i]) + int(n[i]) ** 2].view(int(n[i]), -1))
        one.x_view(0).copy_(bt.X0[int(bt.x_off[i]):int(bt.x_off[i]) + int(n[i] * r[i])].view(int(n[i]), -1))
        g1 = S.Graph()
        Bt.insert(g1, one, [tiles[i]], split=True)
        assert g1.run()[0] == 0
        assert torch.equal(one.a_view(0), bt.a_view(i)) and torch.equal(one.x_view(0), bt.x_view(i))
        g1.close()
    best, table = Bt.autotune([96, 320], copies=8, split=True)
    assert set(best) == {96, 320} and all(t > 0 for v in table.values() for t in v.values())
