"""The tensor-core building blocks (tcgen05 kind::tf32 MMA with operands in
shared memory and the accumulator in tensor memory) against a host matrix
product, in plain tf32 and as the three-term split product."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2507_21913_gb300 as hp  # noqa: E402


@pytest.mark.parametrize("n,k", [(16, 8), (48, 40), (64, 16), (128, 64), (112, 24)])
def test_tc_gemm(n, k):
    g = np.random.Generator(np.random.PCG64(n * 100 + k))
    A = g.uniform(-1, 1, (128, k)).astype(np.float32)
    B = g.uniform(-1, 1, (n, k)).astype(np.float32)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    dA = torch.tensor(A, device="cuda:0")
    dB = torch.tensor(B, device="cuda:0")
    D1 = hp.hpfmm_selftest_tc_gemm(dA, dB, split=False).cpu().numpy()
    D3 = hp.hpfmm_selftest_tc_gemm(dA, dB, split=True).cpu().numpy()
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    e1 = np.max(np.abs(D1 - ref) / scale)
    e3 = np.max(np.abs(D3 - ref) / scale)
    assert e1 < 2e-3          # tf32: 10 explicit mantissa bits
    assert e3 < 2e-6          # split: about 21 bits, fp32 accumulation
    assert e3 < e1 / 10       # the split terms are really there
