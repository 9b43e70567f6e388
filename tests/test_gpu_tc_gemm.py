"""The tensor-core split-BF16 product (tcgen05 MMAs into tensor memory) that
the BF16X3 path runs for chains kept in global memory, checked through the
C-ABI test hook against the same split computed on the host: A and B are
rounded to BF16 hi parts (round to nearest even) with BF16 remainders, and
C must equal A_hi B_hi + A_hi B_lo + A_lo B_hi up to FP32 accumulation, for
single and ragged multi-tile shapes and both operand layouts."""
import numpy as np
import pytest

from paper_2303_13403_gb300 import pqmc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    torch.cuda.set_device(0)
    pqmc.load()


def bf16_rn(x):
    """float32 -> the nearest BF16 value (ties to even), as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def split(x):
    hi = bf16_rn(x)
    lo = bf16_rn((x - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


@pytest.mark.parametrize("M,N,K,trans_a", [(128, 256, 64, False), (200, 300, 100, False), (72, 72, 72, True),
                                           (288, 288, 288, True), (162, 40, 21, False)])
def test_tc_split_bf16_product(M, N, K, trans_a):
    import torch
    rng = np.random.default_rng(M * 7 + N + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    dA = torch.tensor(A.T.copy() if trans_a else A, device="cuda")
    dB = torch.tensor(B, device="cuda")
    dC = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32)
    pqmc.test_tc_gemm(M, N, K, dA.data_ptr(), trans_a, dB.data_ptr(), dC.data_ptr())
    Cg = dC.cpu().numpy().astype(np.float64)
    Ah, Al = split(A)
    Bh, Bl = split(B)
    ref = Ah @ Bh + Ah @ Bl + Al @ Bh
    scale = np.abs(Ah) @ np.abs(Bh)
    assert np.all(np.isfinite(Cg))
    assert np.all(np.abs(Cg - ref) <= 4 * K * 2.0 ** -24 * scale + 1e-30)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    assert np.abs(Cg - exact).max() <= 1e-4 * np.abs(exact).max()
