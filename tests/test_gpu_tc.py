"""The tensor-core (tcgen05 + TMEM + TMA) low-precision tile update
C -= A B^T against exact references.

* integer operands in {-1, 0, 1} (exact in BF16 and TF32, FP32 accumulation
  exact below 2^24): the result must be bit-exact;
* random operands already rounded to the low precision: the reference is the
  FP64 product of the same low-precision values; the only difference is the
  FP32 accumulation, bounded by K * 2^-23 * sum|a||b| (stated tolerance).
"""
import ctypes

import numpy as np
import pytest
import torch

from tests._gpu import need_cuda, spx_mod

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    need_cuda()
    return spx_mod()


def to_tf32(x: torch.Tensor) -> torch.Tensor:
    """Round FP32 to TF32 (nearest, ties away) and keep FP32 storage."""
    b = x.contiguous().view(torch.int32)
    b = (b + 0x1000) & ~0x1FFF
    return b.view(torch.float32)


def tc_gemm(S, C, A, B, prec):
    m, n = C.shape
    K = A.shape[1]
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    P = ctypes.c_void_p
    rc = S.lib.spx_tc_gemm_nt(P(C.data_ptr()), C.stride(0), m, n, P(A.data_ptr()), A.stride(0),
                              P(B.data_ptr()), B.stride(0), K, prec, P(err.data_ptr()),
                              P(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("m,n,K", [(128, 128, 64), (256, 384, 512), (200, 130, 96), (64, 512, 520)])
def test_integer_exact(S, prec, m, n, K):
    g = torch.Generator().manual_seed(m * 7 + n + K)
    A = torch.randint(-1, 2, (m, K), generator=g).double()
    B = torch.randint(-1, 2, (n, K), generator=g).double()
    C = torch.randint(-50, 51, (m, n), generator=g).double()
    ref = C - A @ B.T
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    Ad, Bd = A.to(dt).cuda(), B.to(dt).cuda()
    Cd = C.cuda()
    tc_gemm(S, Cd, Ad, Bd, S.BF16 if prec == "bf16" else S.TF32)
    assert torch.equal(Cd.cpu(), ref)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_random_within_fp32_accumulation(S, prec):
    m, n, K = 384, 256, 512
    g = torch.Generator().manual_seed(3)
    A = torch.rand(m, K, generator=g) * 2 - 1
    B = torch.rand(n, K, generator=g) * 2 - 1
    C = (torch.rand(m, n, generator=g) * 2 - 1).double()
    if prec == "bf16":
        Al, Bl = A.to(torch.bfloat16), B.to(torch.bfloat16)
    else:
        Al, Bl = to_tf32(A), to_tf32(B)
    ref = C - Al.double() @ Bl.double().T
    bound = K * 2.0 ** -23 * (Al.double().abs() @ Bl.double().abs().T) + 1e-300
    Cd = C.cuda()
    tc_gemm(S, Cd, Al.cuda(), Bl.cuda(), S.BF16 if prec == "bf16" else S.TF32)
    assert ((Cd.cpu() - ref).abs() <= bound).all()


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("m,n,K", [(2600, 2432, 200), (4096, 4096, 256)])
def test_integer_exact_many_units(S, prec, m, n, K):
    """More 128 x 128 units than SMs: every CTA of the pipelined kernel runs
    several units, reusing both TMEM accumulators and every operand stage
    (ragged last rows and K chunk included); still bit-exact."""
    g = torch.Generator().manual_seed(m + n + K)
    A = torch.randint(-1, 2, (m, K), generator=g).double()
    B = torch.randint(-1, 2, (n, K), generator=g).double()
    C = torch.randint(-50, 51, (m, n), generator=g).double()
    ref = C - A @ B.T
    dt = torch.bfloat16 if prec == "bf16" else torch.float32
    Cd = C.cuda()
    tc_gemm(S, Cd, A.to(dt).cuda(), B.to(dt).cuda(), S.BF16 if prec == "bf16" else S.TF32)
    assert torch.equal(Cd.cpu(), ref)


def test_widening_exact_for_every_float(S):
    """The epilogues widen the FP32 accumulator to FP64 with integer
    operations only (normal, zero, subnormal, infinite and NaN classes from
    the IEEE formats); over all 2^32 FP32 bit patterns the result equals the
    hardware conversion bit for bit (NaN stays NaN)."""
    bad, _ = S.probe(15, 1)
    assert bad == 0.0, bad
