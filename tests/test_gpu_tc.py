"""The tensor-core (tcgen05) GEMM step the seed network's convolutions are
built from, against a reference product of the same BF16 operands in FP64.
Needs a GPU."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osm():
    from paper_2311_16935_gb300 import build

    build.build()
    from paper_2311_16935_gb300 import osmodi

    return osmodi


@pytest.mark.parametrize("N,K", [(16, 16), (32, 64), (48, 96), (64, 256), (128, 32), (256, 16)])
def test_tc_gemm_matches_reference(osm, N, K):
    g = torch.Generator(device="cuda").manual_seed(N * 1000 + K)
    A = torch.randn((128, K), device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
    D, err = osm.tc_gemm(A, B)
    torch.cuda.synchronize()
    assert err == 0
    ref = A.double() @ B.double().T
    # BF16 products are exact in FP32; only the FP32 summation order differs
    scale = (A.double().abs() @ B.double().abs().T).max().item()
    assert (D.double() - ref).abs().max().item() <= 1e-6 * scale
