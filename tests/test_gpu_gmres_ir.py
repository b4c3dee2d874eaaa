"""GMRES-based iterative refinement (Carson-Higham; spx_gmres_ir) against the
oracle: from the same low-precision factor, refinement whose correction
equation is solved by FP64 GMRES preconditioned with the factor reaches the
FP64 normwise backward error <= 1e-14 (recomputed by the oracle) in fewer
refinement steps than classical refinement, the device's certified eta equals
the oracle's, and non-convergence would be reported, never hidden."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2308_15964_b300 import inputs
from tests._gpu import need_cuda, spx_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    need_cuda()
    return spx_mod()


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("n,sigma,nrhs", [(2048, 1e-3, 8), (1536, 1e-2, 3), (1000, 1e-3, 1)])
def test_gmres_ir_vs_classical(S, prec, n, sigma, nrhs):
    from paper_2308_15964_b300 import mixed
    p = S.TF32 if prec == "tf32" else S.BF16
    b = 512 if n % 512 == 0 else 256
    A = inputs.spd_matrix(n, sigma, seed=9)
    B = inputs.rhs(n, nrhs, seed=9)
    Xg, _, gi = mixed.gmres_ir_solve(A.cuda(), B.cuda(), b=b, prec=p)
    Xc, _, ci = mixed.mixed_solve(A.cuda(), B.cuda(), b=b, prec=p)
    assert gi["status"] == 0 and ci["status"] == 0
    eta = O.solve_backward_error(A.numpy(), Xg.cpu().numpy(), B.numpy())
    print(f"gmres-ir n={n} sigma={sigma} {prec}: converged={gi['converged']} outer={gi['outer']} "
          f"inner={gi['inner']} eta={eta.max():.3e}; classical {ci['iterations']} iterations")
    assert abs(gi["eta_final"] - eta.max()) <= 1e-6 * eta.max()
    assert gi["converged"], gi
    assert eta.max() <= 1e-14
    if ci["converged"]:
        assert gi["outer"] <= max(2, ci["iterations"])
    assert gi["outer"] <= 5


def test_gmres_ir_rejects_bad_arguments(S):
    import ctypes
    P = ctypes.c_void_p
    res = S.GmresResult()
    assert S.lib.spx_gmres_ir(None, 4, 4, None, None, 1, None, None, None, 0, None,
                              ctypes.byref(res), None) == S.ERR_INVALID_ARG
    assert S.lib.spx_gmres_ir_workspace(64, 17, 30) < 0
    assert S.lib.spx_gmres_ir_workspace(64, 4, 65) < 0


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
@pytest.mark.parametrize("sigma", [1e-4, 1e-5])
def test_gmres_ir_ill_conditioned(S, prec, sigma):
    """kappa ~ 1e4 .. 1e5: kappa u_factor >= 1 for BF16, where classical
    refinement may stall; when the low-precision factorization itself
    succeeds, GMRES-based refinement must still reach eta <= 1e-14 (oracle).
    Both outcomes are printed."""
    from paper_2308_15964_b300 import mixed
    p = S.TF32 if prec == "tf32" else S.BF16
    n = 1024
    A = inputs.spd_matrix(n, sigma, seed=11)
    B = inputs.rhs(n, 4, seed=11)
    Xg, _, gi = mixed.gmres_ir_solve(A.cuda(), B.cuda(), b=256, prec=p, max_inner=60)
    if gi["status"] != 0:
        print(f"ill-conditioned sigma={sigma} {prec}: the low-precision factor is not SPD "
              f"(status {gi['status']}, info {gi.get('info')})")
        assert gi["status"] == S.NOT_SPD
        return
    Xc, _, ci = mixed.mixed_solve(A.cuda(), B.cuda(), b=256, prec=p)
    eta = O.solve_backward_error(A.numpy(), Xg.cpu().numpy(), B.numpy())
    etac = O.solve_backward_error(A.numpy(), Xc.cpu().numpy(), B.numpy())
    print(f"ill-conditioned sigma={sigma} {prec}: gmres-ir converged={gi['converged']} "
          f"outer={gi['outer']} inner={gi['inner']} eta={eta.max():.3e}; classical "
          f"converged={ci['converged']} iterations={ci['iterations']} eta={etac.max():.3e}")
    assert abs(gi["eta_final"] - eta.max()) <= 1e-6 * eta.max()
    assert gi["converged"] and eta.max() <= 1e-14, gi
    if not ci["converged"]:
        assert ci["iterations"] == (30 if p == S.TF32 else 50)
