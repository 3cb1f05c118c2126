"""The integer-unit FP32 <-> FP64 conversions of the FP64-bound kernels
(osmodi_probe_convert) against the hardware's IEEE 754 conversions, bit for
bit: random bit patterns over the whole range, exact ties, the binary32
subnormal and overflow boundaries, zeros, infinities and NaNs.  Needs a GPU."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osm():
    from paper_2311_16935_gb300 import build

    build.build()
    from paper_2311_16935_gb300 import osmodi

    return osmodi


def _f64_cases(rng):
    u = [rng.integers(0, 2 ** 64, size=1 << 20, dtype=np.uint64)]
    # exponents around the binary32 subnormal range, 1 and the overflow edge
    ex = np.concatenate([np.arange(855, 905), np.arange(1015, 1035), np.arange(1140, 1160)]).astype(np.uint64)
    e = rng.choice(ex, size=1 << 18)
    m = rng.integers(0, 2 ** 52, size=e.size, dtype=np.uint64)
    tie = rng.random(e.size) < 0.4
    m = np.where(tie, (m >> np.uint64(29) << np.uint64(29)) | np.uint64(1 << 28), m)  # halfway cases
    sign = rng.integers(0, 2, size=e.size, dtype=np.uint64) << np.uint64(63)
    u.append(sign | (e << np.uint64(52)) | m)
    u.append(np.array([0, 1 << 63, 0x7FF0000000000000, 0xFFF0000000000000, 0x7FF8000000000000, 0x7FF0000000000001,
                       0x47EFFFFFF0000000, 0x47EFFFFFE0000000, 0x47EFFFFFEFFFFFFF, 0x36A0000000000000,
                       0x3690000000000000, 0x3690000000000001, 0x380FFFFFF0000000, 0x380FFFFFEFFFFFFF,
                       0x0000000000000001, 0x3FF0000010000000, 0x3FF0000030000000], dtype=np.uint64))
    return np.concatenate(u).view(np.float64)


def _f32_cases(rng):
    b = [rng.integers(0, 2 ** 32, size=1 << 20, dtype=np.uint64).astype(np.uint32),
         np.arange(0, 1 << 16, dtype=np.uint32), np.arange(0x807F0000, 0x80800010, dtype=np.uint32),
         np.array([0x7F800000, 0xFF800000, 0x7FC00000, 0x7F800001, 0xFFFFFFFF, 0x7F7FFFFF, 0x00800000],
                  dtype=np.uint32)]
    return np.concatenate(b).view(np.float32)


def test_conversions_match_hardware_bit_for_bit(osm):
    rng = np.random.default_rng(2311)
    d = _f64_cases(rng)
    f = _f32_cases(rng)
    n = min(d.size, f.size)
    d, f = d[:n], f[:n]
    dt = torch.from_numpy(d.copy()).cuda()
    ft = torch.from_numpy(f.copy()).cuda()
    f_got, d_got = osm.probe_convert(dt, ft)
    f_ref, d_ref = dt.float(), ft.double()
    torch.cuda.synchronize()
    fg, fr = f_got.cpu().numpy().view(np.uint32), f_ref.cpu().numpy().view(np.uint32)
    dg, dr = d_got.cpu().numpy().view(np.uint64), d_ref.cpu().numpy().view(np.uint64)
    nan_d = np.isnan(d)
    # a NaN rounds to a NaN of the same sign (the payload is not specified)
    assert (fg[~nan_d] == fr[~nan_d]).all(), np.flatnonzero(fg[~nan_d] != fr[~nan_d])[:5]
    assert np.isnan(f_got.cpu().numpy()[nan_d]).all()
    nan_f = np.isnan(f)
    assert (dg[~nan_f] == dr[~nan_f]).all(), np.flatnonzero(dg[~nan_f] != dr[~nan_f])[:5]
    assert np.isnan(d_got.cpu().numpy()[nan_f]).all()


def test_convert_rejects_bad_arguments(osm):
    with pytest.raises(TypeError):
        osm.probe_convert(torch.zeros(4, device="cuda"), torch.zeros(4, device="cuda"))
    f_out, d_out = osm.probe_convert(torch.zeros(0, dtype=torch.float64, device="cuda"),
                                     torch.zeros(0, device="cuda"))
    assert f_out.numel() == 0 and d_out.numel() == 0
