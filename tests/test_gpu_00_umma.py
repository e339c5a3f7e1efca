"""tcgen05 operand-layout check: one 128 x N x K UMMA tile from shared-memory
descriptors (no swizzle, K-major core matrices, shifted start rows) against
an FP32 matmul of the same BF16 values.  Runs first so a layout mismatch
stops the GPU suite before the convolution kernel uses the same layout."""
import pytest
import torch

from paper_2108_13830_gb300.binding import umma_selftest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,K,shift", [(32, 32, 0), (32, 32, 5), (16, 32, 3), (32, 16, 0), (16, 16, 37),
                                     (96, 32, 7), (48, 16, 2), (128, 32, 0)])
def test_umma_tile(N, K, shift):
    g = torch.Generator().manual_seed(N * 100 + K + shift)
    A = torch.randn(128 + shift, K, generator=g).bfloat16().cuda()
    B = torch.randn(N, K, generator=g).bfloat16().cuda()
    D = umma_selftest(A, B, N, K, shift=shift, variant=0)
    torch.cuda.synchronize()
    ref = A[shift:shift + 128].double() @ B.double().T
    err = (D.double() - ref).abs().max().item()
    if err > 1e-3 and N <= 64:      # the exchanged-stride probe stays inside its buffer only for N <= 64
        D1 = umma_selftest(A, B, N, K, shift=shift, variant=1)
        torch.cuda.synchronize()
        err1 = (D1.double() - ref).abs().max().item()
        pytest.fail(f"UMMA layout mismatch: err={err} (variant with LBO/SBO exchanged: {err1})")
    assert err <= 1e-3, err
