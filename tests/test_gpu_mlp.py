"""The BF16 tensor-core (tcgen05) kernels of the learned relaxation surrogate."""
import numpy as np
import pytest

from paper_1006_0549_gb300 import lpdf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1006_0549_gb300 import _build
    _build.build()
    return torch


@pytest.mark.parametrize("M,N,K", [(128, 128, 16), (300, 128, 128), (256, 256, 64), (1, 16, 16), (513, 16, 128)])
def test_tc_gemm_matches_fp32_product_of_the_bf16_values(torch_cuda, M, N, K):
    torch = torch_cuda
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    lpdf.tc_gemm_bf16(A.cuda(), B.cuda(), D)
    ref = A.double().numpy() @ B.double().numpy().T          # products of BF16 values are exact in FP32
    got = D.cpu().numpy().astype(np.float64)
    scale = np.abs(A.double().numpy()) @ np.abs(B.double().numpy()).T
    assert np.all(np.abs(got - ref) <= 1e-6 * scale + 1e-30), float(np.max(np.abs(got - ref) / scale))
