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


CONV_SHAPES = [(8, 16, 64, 32, 32), (4, 8, 128, 8, 16), (4, 9, 130, 8, 16), (6, 10, 64, 48, 48), (5, 7, 256, 32, 32),
               (3, 5, 32, 64, 64), (7, 13, 40, 16, 16), (2, 18, 128, 8, 16), (3, 16, 256, 8, 16), (4, 20, 64, 32, 32),
               (3, 34, 64, 8, 16), (3, 10, 130, 32, 32), (2, 6, 128, 16, 48), (1, 3, 128, 8, 16)]


@pytest.mark.parametrize("shape", CONV_SHAPES)
def test_conv3d_matches_torch(osm, shape):
    """A 3x3x3 convolution of the seed network's kind (BF16 operands, FP32
    accumulation, bias and ReLU) by each kernel path against torch's conv3d
    in FP32 on the same BF16 values: the shapes cover one and two 128-voxel
    row segments, rows shorter than 128 joined through their halo, 8 to 64
    channels and a ragged tail in every axis."""
    D, H, W, cin, cout = shape
    g = torch.Generator(device="cuda").manual_seed(sum(shape))
    x = torch.randn((D, H, W, cin), device="cuda", generator=g).to(torch.bfloat16)
    w = (torch.randn((27, cin, cout), device="cuda", generator=g) / (27 * cin) ** 0.5).to(torch.bfloat16)
    bias = torch.randn((cout,), device="cuda", generator=g) * 0.1
    wt = w.float().reshape(3, 3, 3, cin, cout).permute(4, 3, 0, 1, 2).contiguous()
    ref = torch.nn.functional.conv3d(x.float().permute(3, 0, 1, 2).unsqueeze(0), wt, bias, padding=1)
    ref = torch.relu(ref[0].permute(1, 2, 3, 0))
    scale = ref.abs().max().item()
    outs = {}
    for path in (0, 2, 1):
        y, err = osm.conv3d(x, w, bias, relu=True, path=path)
        torch.cuda.synchronize()
        assert err == 0
        d = (y.float() - ref).abs()
        # the output is rounded to BF16 (2^-8 relative); sums differ in order only
        assert d.max().item() <= 2 ** -7 * scale, (path, d.max().item() / scale,
                                                     [int(v) for v in (d == d.max()).nonzero()[0]])
        outs[path] = y
    assert (outs[0].float() - outs[2].float()).abs().max().item() <= 2 ** -7 * scale


@pytest.mark.parametrize("shape", [(64, 128, 128, 8, 16), (32, 64, 64, 32, 32)])
def test_conv3d_large_without_relu(osm, shape):
    """Layers of the seed network's sizes without the ReLU (which would turn
    a NaN into 0): every output finite and equal to the gathering kernel's.
    With 8 input channels the halo kernel pairs the last tap with zero
    weights whose operand lies past the staged box; that slack must hold
    zeros, not whatever shared memory held before."""
    D, H, W, cin, cout = shape
    g = torch.Generator(device="cuda").manual_seed(sum(shape))
    x = torch.randn((D, H, W, cin), device="cuda", generator=g).to(torch.bfloat16)
    w = (torch.randn((27, cin, cout), device="cuda", generator=g) / (27 * cin) ** 0.5).to(torch.bfloat16)
    bias = torch.randn((cout,), device="cuda", generator=g) * 0.1
    outs = []
    for path in (0, 2):
        y, err = osm.conv3d(x, w, bias, relu=False, path=path)
        torch.cuda.synchronize()
        assert err == 0
        outs.append(y.float())
    assert torch.isfinite(outs[0]).all() and torch.isfinite(outs[1]).all()
    scale = outs[1].abs().max().item()
    assert (outs[0] - outs[1]).abs().max().item() <= 2 ** -7 * scale
