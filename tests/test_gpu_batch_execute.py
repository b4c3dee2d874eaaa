"""spx_batch_execute: independently built graphs in one persistent launch.

Each member's result must be bit-identical to running that graph alone (the
FP64 tile ops are deterministic and the members share no tile), and within
the FP64 tolerance of the oracle; a member whose POTRF fails reports its own
SPX_NOT_SPD with the same column as alone while the other members finish; a
mixed-precision member (tensor-core launch) and FP64 members share one launch.
"""
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


def chol_member(S, n, b, nrhs, seed, bad_col=None):
    from paper_2308_15964_b300 import cholesky
    A = inputs.spd_matrix(n, 1.0, seed=seed)
    if bad_col is not None:
        A[bad_col, bad_col] = -5.0
    X = inputs.rhs(n, nrhs, seed=seed)
    Ad, Xd = A.cuda(), X.cuda()
    g = S.Graph()
    cholesky.cholesky_graph(g, Ad, b, Xd)
    return {"g": g, "kind": "chol", "A": A, "X": X, "Ad": Ad, "Xd": Xd, "b": b}


def gemm_member(S, n, b, seed):
    from paper_2308_15964_b300 import cholesky
    A = inputs.uniform((n, n), seed)
    B = inputs.uniform((n, n), seed + 1)
    C = inputs.uniform((n, n), seed + 2)
    Ad, Bd, Cd = A.cuda(), B.cuda(), C.cuda()
    g = S.Graph()
    cholesky.gemm_graph(g, Ad, Bd, Cd, b)
    return {"g": g, "kind": "gemm", "A": A, "B": B, "C": C, "Ad": Ad, "Bd": Bd, "Cd": Cd, "b": b}


def mixed_member(S, n, b, seed):
    from paper_2308_15964_b300 import mixed
    A = inputs.spd_matrix(n, 1.0, seed=seed)
    X = inputs.rhs(n, 2, seed=seed)
    Ad, Xd = A.cuda(), X.cuda()
    Alo = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    g = S.Graph()
    mixed.factor_graph(g, Ad, Alo, b, Xd, S.TF32)
    return {"g": g, "kind": "mixed", "A": A, "X": X, "Ad": Ad, "Xd": Xd, "Alo": Alo, "b": b}


def restore(m):
    if m["kind"] == "gemm":
        m["Cd"].copy_(m["C"].cuda())
    else:
        m["Ad"].copy_(m["A"].cuda())
        m["Xd"].copy_(m["X"].cuda())
        if "Alo" in m:
            m["Alo"].zero_()


def result(m):
    if m["kind"] == "gemm":
        return m["Cd"].cpu().numpy().copy()
    return np.concatenate([m["Ad"].cpu().numpy().ravel(), m["Xd"].cpu().numpy().ravel()])


def run_alone(S, members):
    out = []
    for m in members:
        restore(m)
        rc, info = m["g"].run()
        torch.cuda.synchronize()
        out.append((rc, info, result(m)))
        m["g"].reset()
    return out


def run_batch(S, members, stats=None):
    for m in members:
        restore(m)
    S.batch_execute([m["g"] for m in members])
    out = []
    for m in members:
        rc, info = m["g"].wait()
        out.append((rc, info, result(m)))
    torch.cuda.synchronize()
    if stats is not None:               # counters of the whole launch, via a member
        stats.update(members[0]["g"].stats())
    for m in members:
        m["g"].reset()
    return out


def test_batch_bit_identical_to_alone(S):
    members = [chol_member(S, 512, 64, 1, 21), chol_member(S, 300, 64, 3, 22),
               gemm_member(S, 320, 64, 31), chol_member(S, 96, 32, 2, 23)]
    alone = run_alone(S, members)
    batched = run_batch(S, members)
    for (rc_a, info_a, r_a), (rc_b, info_b, r_b) in zip(alone, batched):
        assert rc_a == rc_b == 0 and info_a == info_b == 0
        assert np.array_equal(r_a, r_b)
    # and against the oracle
    for m, (_, _, r) in zip(members, batched):
        if m["kind"] == "chol":
            n = m["A"].shape[0]
            L, X = m["A"].numpy().copy(), m["X"].numpy().copy()
            assert O.tiled_cholesky(L, m["b"], X) == 0
            Lg = r[:n * n].reshape(n, n)
            err = np.abs(np.tril(Lg) - np.tril(L)).max() / np.abs(np.tril(L)).max()
            assert err <= 1e-12
            Xg = r[n * n:].reshape(X.shape)
            assert O.solve_backward_error(m["A"].numpy(), Xg, m["X"].numpy()).max() <= 1e-14
        else:
            C = m["C"].numpy().copy()
            assert O.tiled_gemm(m["A"].numpy(), m["B"].numpy(), C, m["b"]) == 0
            n = C.shape[0]
            bound = 4 * n * 2.2e-16 * (np.abs(m["A"].numpy()) @ np.abs(m["B"].numpy())).max()
            assert np.abs(r - C).max() <= bound
    # a second batch of the same graphs (the merged graph is rebuilt), then a
    # member alone again
    again = run_batch(S, members)
    for (_, _, r_a), (_, _, r_b) in zip(alone, again):
        assert np.array_equal(r_a, r_b)
    restore(members[1])
    assert members[1]["g"].run()[0] == 0
    assert np.array_equal(result(members[1]), alone[1][2])
    for m in members:
        m["g"].close()


def test_failing_member_is_isolated(S):
    members = [chol_member(S, 256, 64, 1, 41), chol_member(S, 192, 64, 1, 42, bad_col=100),
               chol_member(S, 256, 64, 2, 43)]
    alone = run_alone(S, members)
    assert alone[1][0] == S.NOT_SPD and alone[1][1] == 101
    batched = run_batch(S, members)
    assert batched[1][0] == S.NOT_SPD and batched[1][1] == 101
    for i in (0, 2):
        assert batched[i][0] == 0 and np.array_equal(batched[i][2], alone[i][2])
    for m in members:
        m["g"].close()


def test_mixed_and_fp64_members_share_a_launch(S):
    members = [mixed_member(S, 512, 128, 51), chol_member(S, 384, 64, 2, 52)]
    alone = run_alone(S, members)
    st = {}
    batched = run_batch(S, members, stats=st)
    for (rc_a, _, r_a), (rc_b, _, r_b) in zip(alone, batched):
        assert rc_a == rc_b == 0
        assert np.array_equal(r_a, r_b)
    assert st["parts"] > 0 and "SYRK" in st["op_cycles"] and "TRSM" in st["op_cycles"]
    for m in members:
        m["g"].close()
