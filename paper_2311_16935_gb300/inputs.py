"""Seeded synthetic inputs: pressure-gradient fields, masks and noise.

This module holds none of the integration method's arithmetic.  It only
builds the data the solver and the CPU oracle both consume: analytic
gradients of known pressure fields, validity masks and Gaussian noise, all
drawn from seeded generators so that every run sees the same inputs.

Conventions shared with the solver's C interface: a 2D field has shape
(ny, nx), a 3D field (nz, ny, nx), x fastest; a gradient field has one extra
leading axis holding the components (x first).  Masks are uint8, nonzero =
data available.

Workloads (the paper measures on JHU turbulence cut-outs and PIV
experiments that are not available here; these synthetic fields stand in
with the same shapes and the same kinds of structure):

* ``lamb_oseen_2d``   64 x 64 on [0,1]^2, Lamb-Oseen vortex, 2 % noise, FP64
* ``sincos_3d``       128^3 on [0, 2 pi]^3, smooth trigonometric field,
                      spherical solid mask of radius 0.5 at the centre, 5 % noise
* ``piv_batch_2d``    512 snapshots of uneven sizes (128..1024 x 128..512),
                      0-3 elliptical solid masks each, Taylor-Green-like field,
                      1-5 % noise
* ``gaussian_blobs_3d`` 500^3 (or any box), 20 random Gaussian pressure blobs,
                      3 % noise
Noise is i.i.d. N(0, sigma^2) on every gradient component at every point with
sigma = s * max over valid points of |grad p|.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch


def _rng(*key) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


def _noise_like(g: torch.Tensor, sigma: float, seed) -> torch.Tensor:
    gen = torch.Generator(device=g.device)
    gen.manual_seed(int(np.random.SeedSequence(list(seed)).generate_state(1, np.uint64)[0] & 0x7FFFFFFFFFFFFFFF))
    return torch.randn(g.shape, generator=gen, device=g.device, dtype=torch.float64) * sigma


@dataclass
class Problem:
    """One solve's inputs: gradient (ndim, *shape), mask (*shape) uint8,
    spacing per axis (x first), and the analytic pressure if known."""

    grad: torch.Tensor
    mask: torch.Tensor
    spacing: tuple
    p_true: torch.Tensor | None = None
    meta: dict = field(default_factory=dict)

    @property
    def ndim(self) -> int:
        return self.mask.dim()

    @property
    def dims(self) -> tuple:
        return tuple(self.mask.shape[::-1])


def _max_valid_norm(g: torch.Tensor, mask: torch.Tensor) -> float:
    mag = torch.sqrt((g * g).sum(0))
    mag = torch.where(mask.bool(), mag, torch.zeros_like(mag))
    return float(mag.max())


# --------------------------------------------------------------------------
# Analytic fields
# --------------------------------------------------------------------------

def quadratic_field(shape, spacing, coeffs=None, seed=0, device="cpu"):
    """p = a0 + a.x + x^T B x (any ndim) with its exact gradient.  The
    trapezoidal face average of a linear gradient is exact, so this p is an
    exact fixed point of the method for any mask and spacing."""
    ndim = len(shape)
    rng = _rng(17, seed)
    if coeffs is None:
        lin = rng.normal(size=ndim)
        B = rng.normal(size=(ndim, ndim))
        B = 0.5 * (B + B.T)
    else:
        lin, B = coeffs
    axes = [torch.arange(n, dtype=torch.float64, device=device) * spacing[ndim - 1 - q]
            for q, n in enumerate(shape)]
    grids = torch.meshgrid(*axes, indexing="ij")  # grids[q] varies along array axis q
    X = [grids[ndim - 1 - a] for a in range(ndim)]  # X[a] = coordinate along physical axis a
    p = torch.zeros(shape, dtype=torch.float64, device=device) + 0.3
    g = torch.zeros((ndim,) + tuple(shape), dtype=torch.float64, device=device)
    for a in range(ndim):
        p = p + lin[a] * X[a]
        g[a] += lin[a]
        for b in range(ndim):
            p = p + B[a, b] * X[a] * X[b]
            g[a] += 2.0 * B[a, b] * X[b]
    return p, g


def lamb_oseen_2d(n=64, noise=0.02, seed=1, rc=0.1, gamma=1.0, rho=1.0, device="cpu") -> Problem:
    """n x n nodes on [0,1]^2 (spacing 1/(n-1)), Lamb-Oseen vortex centred at
    (0.5, 0.5): u_theta = Gamma/(2 pi r) (1 - exp(-r^2/rc^2)), dp/dr =
    rho u_theta^2 / r, plus Gaussian noise.  No mask."""
    h = 1.0 / (n - 1)
    x = torch.arange(n, dtype=torch.float64, device=device) * h
    Y, X = torch.meshgrid(x, x, indexing="ij")
    dx, dy = X - 0.5, Y - 0.5
    r = torch.sqrt(dx * dx + dy * dy)
    rs = torch.where(r > 0, r, torch.ones_like(r))  # a node on the centre (odd n): gradient 0 there
    ut = gamma / (2 * math.pi * rs) * (1 - torch.exp(-rs * rs / (rc * rc)))
    dpdr = rho * ut * ut / rs
    g = torch.stack([dpdr * dx / rs, dpdr * dy / rs])
    g = torch.where(r > 0, g, torch.zeros_like(g))
    mask = torch.ones((n, n), dtype=torch.uint8, device=device)
    sigma = noise * _max_valid_norm(g, mask)
    g = g + _noise_like(g, sigma, (1, seed))
    return Problem(g, mask, (h, h), None, dict(workload=f"lamb_oseen_2d_{n}x{n}", noise=noise))


def sincos_3d(n=128, noise=0.05, seed=2, mask_radius=0.5, dtype=torch.float32, device="cpu") -> Problem:
    """n^3 nodes on [0, 2 pi]^3 (spacing 2 pi/(n-1)); p = sin x cos y sin z +
    0.5 cos 2x sin z with its analytic gradient; cells strictly inside the
    sphere of radius mask_radius about (pi, pi, pi) are masked out."""
    h = 2 * math.pi / (n - 1)
    x = torch.arange(n, dtype=torch.float64, device=device) * h
    Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")
    p = torch.sin(X) * torch.cos(Y) * torch.sin(Z) + 0.5 * torch.cos(2 * X) * torch.sin(Z)
    gx = torch.cos(X) * torch.cos(Y) * torch.sin(Z) - torch.sin(2 * X) * torch.sin(Z)
    gy = -torch.sin(X) * torch.sin(Y) * torch.sin(Z)
    gz = torch.sin(X) * torch.cos(Y) * torch.cos(Z) + 0.5 * torch.cos(2 * X) * torch.cos(Z)
    g = torch.stack([gx, gy, gz])
    c = math.pi
    inside = (X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2 < mask_radius**2
    mask = (~inside).to(torch.uint8)
    sigma = noise * _max_valid_norm(g, mask)
    g = g + _noise_like(g, sigma, (2, seed))
    return Problem(g.to(dtype), mask, (h, h, h), p, dict(workload=f"sincos_3d_{n}^3_sphere_mask", noise=noise))


def _ellipse_mask(nx, ny, hx, hy, rng, n_ell):
    Lx, Ly = (nx - 1) * hx, (ny - 1) * hy
    x = np.arange(nx) * hx
    y = np.arange(ny) * hy
    Xg, Yg = np.meshgrid(x, y)
    mask = np.ones((ny, nx), dtype=np.uint8)
    ext = min(Lx, Ly)
    for _ in range(n_ell):
        cx, cy = rng.uniform(0, Lx), rng.uniform(0, Ly)
        a, b = rng.uniform(0.05, 0.2) * ext, rng.uniform(0.05, 0.2) * ext
        th = rng.uniform(0, math.pi)
        u = (Xg - cx) * math.cos(th) + (Yg - cy) * math.sin(th)
        v = -(Xg - cx) * math.sin(th) + (Yg - cy) * math.cos(th)
        mask[(u / a) ** 2 + (v / b) ** 2 < 1.0] = 0
    return mask


def piv_snapshot_2d(index: int, base_seed: int = 3, size_range=((128, 1024), (128, 512)), device="cpu",
                    dtype=torch.float32) -> Problem:
    """One snapshot of the batched PIV-like workload: nx ~ U{128..1024},
    ny ~ U{128..512}; spacing 1/(nx-1) on both axes; p = a/4 [cos(2 pi kx x) +
    cos(2 pi ky y / Ly)], kx, ky ~ U{1..8}; 0-3 elliptical solid masks
    (semi-axes 0.05-0.2 of the smaller extent, redrawn if fewer than half the
    cells stay valid); noise s ~ U[0.01, 0.05]."""
    rng = _rng(base_seed, index)
    (nx_lo, nx_hi), (ny_lo, ny_hi) = size_range
    nx = int(rng.integers(nx_lo, nx_hi + 1))
    ny = int(rng.integers(ny_lo, ny_hi + 1))
    h = 1.0 / (nx - 1)
    kx, ky = int(rng.integers(1, 9)), int(rng.integers(1, 9))
    s = float(rng.uniform(0.01, 0.05))
    n_ell = int(rng.integers(0, 4))
    while True:
        mask_np = _ellipse_mask(nx, ny, h, h, rng, n_ell)
        if mask_np.mean() >= 0.5:
            break
    Ly = (ny - 1) * h
    x = torch.arange(nx, dtype=torch.float64, device=device) * h
    y = torch.arange(ny, dtype=torch.float64, device=device) * h
    Y, X = torch.meshgrid(y, x, indexing="ij")
    a = 1.0
    p = 0.25 * a * (torch.cos(2 * math.pi * kx * X) + torch.cos(2 * math.pi * ky * Y / Ly))
    gx = -0.25 * a * 2 * math.pi * kx * torch.sin(2 * math.pi * kx * X)
    gy = -0.25 * a * 2 * math.pi * ky / Ly * torch.sin(2 * math.pi * ky * Y / Ly)
    g = torch.stack([gx, gy])
    mask = torch.from_numpy(mask_np).to(device)
    sigma = s * _max_valid_norm(g, mask)
    g = g + _noise_like(g, sigma, (base_seed, index, 99))
    return Problem(g.to(dtype), mask, (h, h), p, dict(workload="piv_batch_2d", noise=s, n_ellipses=n_ell))


def piv_batch_2d(count=512, base_seed=3, device="cpu", dtype=torch.float32, **kw):
    return [piv_snapshot_2d(i, base_seed, device=device, dtype=dtype, **kw) for i in range(count)]


def blob_params(n_blobs=20, box=(500, 500, 500), width_range=(5.0, 40.0), seed=4):
    rng = _rng(seed, 0)
    centres = np.stack([rng.uniform(0, box[a] - 1, size=n_blobs) for a in range(3)], axis=1)  # x, y, z
    amps = rng.normal(size=n_blobs)
    widths = rng.uniform(width_range[0], width_range[1], size=n_blobs)
    return centres, amps, widths


def gaussian_blobs_3d(n=(500, 500, 500), noise=0.03, seed=4, n_blobs=20, width_range=(5.0, 40.0),
                      origin=(0, 0, 0), box=None, device="cpu", dtype=torch.float32, with_pressure=False,
                      params=None, chunk_planes=16) -> Problem:
    """Sum of Gaussian pressure blobs on a box of n = (nx, ny, nz) cells with
    unit spacing: p = sum_b a_b exp(-|x - c_b|^2 / (2 w_b^2)), a_b ~ N(0,1),
    w_b ~ U[5, 40] cells, centres uniform in ``box`` (default: the grid
    itself).  ``origin`` offsets the grid inside the box (crops).  The
    gradient is analytic; noise sigma = noise * max |grad p| over the grid.
    Built plane-chunk by plane-chunk so that 500^3 fits comfortably."""
    nx, ny, nz = n
    if box is None:
        box = n
    centres, amps, widths = params if params is not None else blob_params(n_blobs, box, width_range, seed)
    g = torch.empty((3, nz, ny, nx), dtype=dtype, device=device)
    p_out = torch.empty((nz, ny, nx), dtype=torch.float64, device=device) if with_pressure else None
    x = torch.arange(nx, dtype=torch.float64, device=device) + origin[0]
    y = torch.arange(ny, dtype=torch.float64, device=device) + origin[1]
    gmax = 0.0
    for z0 in range(0, nz, chunk_planes):
        z1 = min(nz, z0 + chunk_planes)
        z = torch.arange(z0, z1, dtype=torch.float64, device=device) + origin[2]
        Z, Y, X = torch.meshgrid(z, y, x, indexing="ij")
        gx = torch.zeros_like(X)
        gy = torch.zeros_like(X)
        gz = torch.zeros_like(X)
        pp = torch.zeros_like(X) if with_pressure else None
        for b in range(len(amps)):
            dx, dy, dz = X - centres[b, 0], Y - centres[b, 1], Z - centres[b, 2]
            e = amps[b] * torch.exp(-(dx * dx + dy * dy + dz * dz) / (2 * widths[b] ** 2))
            s = -1.0 / widths[b] ** 2
            gx += s * dx * e
            gy += s * dy * e
            gz += s * dz * e
            if with_pressure:
                pp += e
        gmax = max(gmax, float(torch.sqrt(gx * gx + gy * gy + gz * gz).max()))
        g[0, z0:z1] = gx.to(dtype)
        g[1, z0:z1] = gy.to(dtype)
        g[2, z0:z1] = gz.to(dtype)
        if with_pressure:
            p_out[z0:z1] = pp
        del gx, gy, gz, X, Y, Z
    sigma = noise * gmax
    if sigma > 0:
        gen = torch.Generator(device=g.device)
        gen.manual_seed(int(np.random.SeedSequence([seed, 7]).generate_state(1, np.uint64)[0] & 0x7FFFFFFFFFFFFFFF))
        for a in range(3):
            for z0 in range(0, nz, chunk_planes):
                z1 = min(nz, z0 + chunk_planes)
                nz_ = torch.randn((z1 - z0, ny, nx), generator=gen, device=g.device, dtype=torch.float32)
                g[a, z0:z1] += (nz_ * sigma).to(dtype)
    mask = torch.ones((nz, ny, nx), dtype=torch.uint8, device=device)
    return Problem(g, mask, (1.0, 1.0, 1.0), p_out,
                   dict(workload=f"gaussian_blobs_3d_{nx}x{ny}x{nz}", noise=noise, sigma=sigma))


def random_mask(shape, p_missing=0.2, seed=0, device="cpu"):
    """Independent per-cell missing data (for edge-case tests)."""
    rng = _rng(23, seed)
    return torch.from_numpy((rng.random(shape) >= p_missing).astype(np.uint8)).to(device)


def random_gradient(shape, seed=0, dtype=torch.float64, device="cpu"):
    """A generic (non curl-free) gradient field with N(0,1) components."""
    rng = _rng(29, seed)
    ndim = len(shape)
    return torch.from_numpy(rng.normal(size=(ndim,) + tuple(shape))).to(device=device, dtype=dtype)
