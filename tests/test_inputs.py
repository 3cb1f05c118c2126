"""The seeded input generators against the recipe they state (shapes, value
distributions, masks, noise level, determinism, crops).  CPU only."""
import math

import numpy as np
import pytest
import torch

from paper_2311_16935_gb300 import inputs


def _max_norm(g, mask):
    mag = torch.sqrt((g.double() ** 2).sum(0))
    return float(mag[mask.bool()].max())


def test_seeded_generators_are_deterministic():
    a = inputs.piv_snapshot_2d(5)
    b = inputs.piv_snapshot_2d(5)
    c = inputs.piv_snapshot_2d(6)
    assert torch.equal(a.grad, b.grad) and torch.equal(a.mask, b.mask)
    assert a.grad.shape != c.grad.shape or not torch.equal(a.grad, c.grad)
    assert torch.equal(inputs.lamb_oseen_2d().grad, inputs.lamb_oseen_2d().grad)
    assert torch.equal(inputs.random_mask((7, 9), seed=3), inputs.random_mask((7, 9), seed=3))


def test_lamb_oseen_recipe():
    prob = inputs.lamb_oseen_2d(n=64)
    clean = inputs.lamb_oseen_2d(n=64, noise=0.0)
    assert prob.grad.shape == (2, 64, 64) and prob.grad.dtype == torch.float64
    assert prob.mask.all() and prob.spacing == pytest.approx((1 / 63, 1 / 63))
    sigma = 0.02 * _max_norm(clean.grad, clean.mask)
    noise = (prob.grad - clean.grad).numpy().ravel()
    assert abs(noise.mean()) < 4 * sigma / math.sqrt(noise.size)
    assert noise.std() == pytest.approx(sigma, rel=0.03)
    # the clean field is the radial pressure gradient of the vortex: tangential
    # component zero (g . t = 0 with t = (-dy, dx))
    h = 1 / 63
    x = torch.arange(64, dtype=torch.float64) * h
    Y, X = torch.meshgrid(x, x, indexing="ij")
    tang = clean.grad[0] * -(Y - 0.5) + clean.grad[1] * (X - 0.5)
    assert float(tang.abs().max()) < 1e-12


def test_sincos_mask_and_noise():
    n = 33
    prob = inputs.sincos_3d(n=n, noise=0.05)
    clean = inputs.sincos_3d(n=n, noise=0.0, dtype=torch.float64)
    assert prob.grad.dtype == torch.float32 and prob.grad.shape == (3, n, n, n)
    h = 2 * math.pi / (n - 1)
    idx = np.arange(n) * h - math.pi
    Z, Y, X = np.meshgrid(idx, idx, idx, indexing="ij")
    inside = X ** 2 + Y ** 2 + Z ** 2 < 0.25
    assert np.array_equal(prob.mask.numpy() == 0, inside)
    sigma = 0.05 * _max_norm(clean.grad, clean.mask)
    noise = (prob.grad.double() - clean.grad).numpy().ravel()
    assert noise.std() == pytest.approx(sigma, rel=0.03)
    # analytic gradient: central differences of p agree to O(h^2)
    p = clean.p_true.numpy()
    gx = (p[:, :, 2:] - p[:, :, :-2]) / (2 * h)
    assert np.abs(gx - clean.grad[0].numpy()[:, :, 1:-1]).max() < 2.0 * h * h


def test_piv_snapshot_recipe():
    sizes, ells = [], []
    for i in range(24):
        prob = inputs.piv_snapshot_2d(i)
        ny, nx = prob.mask.shape
        assert 128 <= nx <= 1024 and 128 <= ny <= 512
        assert prob.grad.shape == (2, ny, nx) and prob.grad.dtype == torch.float32
        assert prob.spacing == pytest.approx((1 / (nx - 1), 1 / (nx - 1)))
        assert 0 <= prob.meta["n_ellipses"] <= 3 and 0.01 <= prob.meta["noise"] <= 0.05
        assert float(prob.mask.double().mean()) >= 0.5
        if prob.meta["n_ellipses"] == 0:
            assert prob.mask.all()
        sizes.append(nx * ny)
        ells.append(prob.meta["n_ellipses"])
    assert len(set(sizes)) > 20 and len(set(ells)) >= 3  # uneven sizes, varied masks


def test_blob_field_analytic_chunking_and_crop():
    n = (24, 20, 18)
    params = inputs.blob_params(20, n, (5.0, 40.0), 4)
    full = inputs.gaussian_blobs_3d(n=n, noise=0.0, params=params, dtype=torch.float64, with_pressure=True,
                                    chunk_planes=16)
    chunked = inputs.gaussian_blobs_3d(n=n, noise=0.0, params=params, dtype=torch.float64, chunk_planes=5)
    assert torch.equal(full.grad, chunked.grad)
    # analytic gradient: central differences of the stored pressure, O(h^2)
    # with widths of at least 5 cells
    p = full.p_true.numpy()
    for a, sl in ((0, np.s_[:, :, 1:-1]), (1, np.s_[:, 1:-1, :]), (2, np.s_[1:-1, :, :])):
        d = np.gradient(p, axis=2 - a)[sl]
        assert np.abs(d - full.grad[a].numpy()[sl]).max() < 0.05 * np.abs(full.grad[a].numpy()).max()
    # a crop with an origin offset is the same field's sub-block (the CPU
    # baseline's 100^3 crop of the 500^3 workload relies on it)
    crop = inputs.gaussian_blobs_3d(n=(8, 6, 5), origin=(10, 7, 4), box=n, noise=0.0, params=params,
                                    dtype=torch.float64)
    assert torch.allclose(crop.grad, full.grad[:, 4:9, 7:13, 10:18], rtol=0, atol=1e-15)


def test_blob_noise_level():
    n = (40, 36, 32)
    clean = inputs.gaussian_blobs_3d(n=n, noise=0.0, dtype=torch.float64)
    noisy = inputs.gaussian_blobs_3d(n=n, noise=0.03, dtype=torch.float64)
    sigma = noisy.meta["sigma"]
    assert sigma == pytest.approx(0.03 * _max_norm(clean.grad, clean.mask), rel=1e-12)
    d = (noisy.grad - clean.grad).numpy().ravel()
    assert d.std() == pytest.approx(sigma, rel=0.02)


def test_quadratic_field_is_exact():
    p, g = inputs.quadratic_field((9, 11, 13), (0.5, 0.7, 1.1), seed=2)
    h = {0: 0.5, 1: 0.7, 2: 1.1}
    for a in range(3):  # physical axis a is array axis 2 - a
        ax = 2 - a
        d = (np.take(p.numpy(), range(2, p.shape[ax]), axis=ax) - np.take(p.numpy(), range(0, p.shape[ax] - 2), axis=ax))
        d /= 2 * h[a]
        ref = np.take(g[a].numpy(), range(1, p.shape[ax] - 1), axis=ax)
        assert np.abs(d - ref).max() < 1e-11  # central differences are exact on quadratics
