"""GPU parity of the paper's other two test cases on the same engine
(section "Numerical applications"):

* AXPY in single precision, the vector split into independent pieces: bit-exact
  against the oracle's FP32 loop (one rounding per operation on both sides),
  for pieces that are multiples of 1024 (tiles of 1024 columns), ragged
  pieces (one row), and several alphas;
* particle interactions (direct Coulomb sum, FP64, dependencies on whole
  groups): within the FP64 summation bound of the oracle for WRITE and
  COMMUTATIVE_WRITE task lists; the closed forms (two charges; six charges
  around the origin) exactly; WRITE runs bit-identical across executors.
"""
import ctypes

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


@pytest.mark.parametrize("n,piece,alpha", [((1 << 20) + 12345, 4096, 1.0),
                                           ((1 << 20) + 12345, 1 << 18, 0.5),
                                           (100000, 1000, -3.25), (5000, 5000, 1.1),
                                           (1 << 22, 1 << 22, 2.0)])
def test_axpy_bit_exact(S, n, piece, alpha):
    x = inputs.uniform((n,), 21).numpy().astype(np.float32)
    y = inputs.uniform((n,), 22).numpy().astype(np.float32)
    yo = y.copy()
    O.axpy_f32(x, yo, alpha)
    dx, dy = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    g = S.Graph()
    nt = ctypes.c_longlong()
    assert S.lib.spx_axpy_insert(g._h, ctypes.c_void_p(dx.data_ptr()),
                                 ctypes.c_void_p(dy.data_ptr()), n, piece, alpha,
                                 ctypes.byref(nt)) == 0
    assert nt.value == -(-n // piece)
    g.derive()
    assert g.sizes()[1] == 0                 # independent pieces: no edges
    assert g.run()[0] == 0
    assert np.array_equal(dy.cpu().numpy(), yo)
    g.close()


def particle_groups(sizes, seed):
    N = int(np.sum(sizes))
    P = np.zeros((N, 8), np.float64)
    P[:, 0:3] = inputs.uniform((N, 3), seed).numpy()
    P[:, 3] = inputs.uniform((N,), seed + 1).numpy()
    return P


def run_nbody(S, P, sizes, commutative=False, executor=0):
    from paper_2308_15964_b300 import spx
    dP = torch.from_numpy(P.copy()).cuda()
    offs = np.concatenate([[0], np.cumsum(sizes)])
    ptrs = (ctypes.c_void_p * len(sizes))(*[dP.data_ptr() + 8 * 8 * int(o) for o in offs[:-1]])
    sz = (ctypes.c_int * len(sizes))(*[int(v) for v in sizes])
    g = S.Graph(executor=executor)
    nt = ctypes.c_longlong()
    assert S.lib.spx_nbody_insert(g._h, len(sizes), ptrs, sz, 1 if commutative else 0,
                                  ctypes.byref(nt)) == 0
    assert nt.value == len(sizes) * (len(sizes) + 1) // 2
    assert g.run()[0] == 0
    out = dP.cpu().numpy()
    g.close()
    return out


def test_nbody_closed_forms(S):
    P = np.zeros((2, 8))
    P[0, 3], P[1, 0], P[1, 3] = 2.0, 2.0, 3.0
    out = run_nbody(S, P, [2])
    assert out[0, 4] == 1.5 and out[1, 4] == 1.0
    assert out[0, 5] == -0.75 and out[1, 5] == 0.5 and not out[:, 6:].any()
    Q = np.zeros((7, 8))
    Q[0, 3] = 1.0
    for k, (ax, sg) in enumerate([(0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1)]):
        Q[k + 1, ax] = sg
        Q[k + 1, 3] = 1.0
    for sizes in ([7], [3, 4]):
        out = run_nbody(S, Q, sizes)
        assert out[0, 4] == 6.0 and not out[0, 5:].any()


@pytest.mark.parametrize("sizes", [[300], [100, 37, 256, 1, 64], [64] * 9, [513, 1000]])
@pytest.mark.parametrize("commutative", [False, True])
def test_nbody_vs_oracle(S, sizes, commutative):
    P = particle_groups(sizes, 31 + len(sizes))
    Po = P.copy()
    assert O.nbody(Po, sizes) == 0
    got = run_nbody(S, P, sizes, commutative)
    assert np.array_equal(got[:, :4], P[:, :4])          # inputs untouched
    X, q = P[:, :3], P[:, 3]
    d = X[:, None, :] - X[None, :, :]
    r2 = (d ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    # FP64 summation bound: a few ulps per term times the number of terms
    bound_phi = 8 * len(q) * 2.2e-16 * (np.abs(q)[None, :] / np.sqrt(r2)).sum(1)
    bound_E = 8 * len(q) * 2.2e-16 * (np.abs(q)[None, :] / r2).sum(1)
    assert (np.abs(got[:, 4] - Po[:, 4]) <= bound_phi).all()
    assert (np.abs(got[:, 5:] - Po[:, 5:]) <= bound_E[:, None]).all()


def test_nbody_executors_bit_identical(S):
    sizes = [90, 200, 33, 128]
    P = particle_groups(sizes, 77)
    outs = [run_nbody(S, P, sizes, False, ex) for ex in (S.EXEC_PERSISTENT, S.EXEC_PER_TASK,
                                                          S.EXEC_STREAMS)]
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
