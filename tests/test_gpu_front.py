"""The source-term front-end kernels against the FP64 oracle, element by
element, on masked grids that exercise every case of the difference rule,
and one velocity-to-pressure pipeline with an exact answer.  Needs a GPU."""
import numpy as np
import pytest
import torch

import oracle
from oracle import front

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osm():
    from paper_2311_16935_gb300 import build

    build.build()
    from paper_2311_16935_gb300 import osmodi

    return osmodi


CASES = [((23, 37), (0.1, 0.13)), ((5, 130), (1.0, 1.0)), ((6, 9, 14), (0.5, 0.7, 0.4)), ((11, 5, 33), (1.0, 1.0, 1.0))]


def _setup(osm, shape, spacing, seed, drop=0.25):
    rng = np.random.default_rng(seed)
    valid = rng.random(shape) > drop
    nd = len(shape)
    plan = osm.Plan(nd, shape[::-1], spacing, torch.from_numpy(valid.astype(np.uint8)).cuda())
    return rng, valid, plan


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _cuda(a):
    return torch.from_numpy(_f32(a)).cuda()


def _close(got, want, valid):
    """FP32 arithmetic on FP32 inputs against FP64 on the same inputs."""
    scale = np.abs(want).max()
    np.testing.assert_allclose(got[:, valid], want[:, valid], rtol=0, atol=2e-5 * scale)
    assert np.all(got[:, ~valid] == 0.0)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("tmode", ["steady", "prev", "next", "both"])
def test_incompressible_matches_oracle(osm, case, tmode):
    shape, spacing = CASES[case]
    rng, valid, plan = _setup(osm, shape, spacing, 30 + case)
    nd = len(shape)
    u = _f32(rng.normal(size=(nd,) + shape))
    up = _f32(u + 0.1 * rng.normal(size=u.shape)) if tmode in ("prev", "both") else None
    un = _f32(u + 0.1 * rng.normal(size=u.shape)) if tmode in ("next", "both") else None
    dt, rho, mu = 0.05, 1.2, 0.03
    got = plan.source_incompressible(_cuda(u), None if up is None else _cuda(up), None if un is None else _cuda(un),
                                     dt=dt, rho=rho, mu=mu).cpu().numpy()
    want = front.incompressible(valid, spacing, u, up, un, dt=dt, rho=rho, mu=mu)
    _close(got, want, valid)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_rans_matches_oracle(osm, case):
    shape, spacing = CASES[case]
    rng, valid, plan = _setup(osm, shape, spacing, 40 + case)
    nd = len(shape)
    U = _f32(rng.normal(size=(nd,) + shape))
    R = _f32(0.3 * rng.normal(size=(3 if nd == 2 else 6,) + shape))
    got = plan.source_rans(_cuda(U), _cuda(R), rho=0.9).cpu().numpy()
    want = front.rans(valid, spacing, U, R, rho=0.9)
    _close(got, want, valid)


def _psd_stress(rng, nd, shape, scale):
    """Per-cell covariance matrices (physical Reynolds stresses)."""
    B = rng.normal(size=(nd, nd) + shape) * scale
    C = np.einsum("ik...,jk...->ij...", B, B)
    if nd == 2:
        return np.stack([C[0, 0], C[1, 1], C[0, 1]])
    return np.stack([C[0, 0], C[1, 1], C[2, 2], C[0, 1], C[0, 2], C[1, 2]])


@pytest.mark.parametrize("case", range(len(CASES)))
def test_compressible_matches_oracle(osm, case):
    shape, spacing = CASES[case]
    rng, valid, plan = _setup(osm, shape, spacing, 50 + case)
    nd = len(shape)
    consts = (1.4, 0.7, 230.0, 260.0, 287.0)
    U = _f32(230.0 * (1.0 + 0.2 * rng.normal(size=(nd,) + shape)))
    R = _f32(_psd_stress(rng, nd, shape, 20.0))
    g, T = plan.source_compressible(_cuda(U), _cuda(R), *consts)
    want, Tw = front.compressible(valid, spacing, U, R, *consts)
    _close(g.cpu().numpy(), want, valid)
    np.testing.assert_allclose(T.cpu().numpy()[valid], Tw[valid], rtol=1e-5)


def test_velocity_to_pressure_pipeline_exact(osm):
    """Plane stagnation flow U = a (x - xc, -(y - yc)), R = 0, two solid
    bodies: the RANS source is exactly grad p with p = -rho a^2 r^2 / 2, and
    the integration (FP32 sweeps, FP64 refinement) returns p up to a
    constant to FP32-input accuracy."""
    nx, ny, hx, hy, rho, a = 301, 203, 0.01, 0.012, 1.1, 1.5
    y, x = np.meshgrid(np.arange(ny) * hy, np.arange(nx) * hx, indexing="ij")
    valid = np.ones((ny, nx), bool)
    for cx, cy, r in [(1.0, 1.2, 0.3), (2.2, 0.8, 0.25)]:
        valid &= (x - cx) ** 2 + (y - cy) ** 2 > r * r
    xc, yc = 1.5, 1.2
    U = np.stack([a * (x - xc), -a * (y - yc)])
    p = -rho * a * a * ((x - xc) ** 2 + (y - yc) ** 2) / 2
    plan = osm.Plan(2, (nx, ny), (hx, hy), torch.from_numpy(valid.astype(np.uint8)).cuda())
    f = plan.source_rans(_cuda(U), torch.zeros((3, ny, nx), dtype=torch.float32, device="cuda"), rho=rho)
    P = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
    res = plan.solve(f, P, 1e-10)
    assert res.status == osm.OK
    grid = oracle.Grid(valid, (hx, hy))
    want = oracle.gauge(grid, np.where(valid, p, np.nan))
    got = P.cpu().numpy()
    assert np.linalg.norm(got[valid] - want[valid]) <= 1e-5 * np.linalg.norm(want[valid])


def test_front_end_argument_errors(osm):
    plan = osm.Plan(2, (8, 6), (1.0, 1.0), None)
    u = torch.zeros((2, 6, 8), dtype=torch.float32, device="cuda")
    lib = osm.lib()
    out = torch.empty_like(u)
    assert lib.osmodi_source_incompressible(plan.handle, None, None, None, 1.0, 1.0, 0.0, out.data_ptr(), None) == osm.E_INVALID
    # a neighbour snapshot needs dt > 0
    assert lib.osmodi_source_incompressible(plan.handle, u.data_ptr(), u.data_ptr(), None, 0.0, 1.0, 0.0,
                                            out.data_ptr(), None) == osm.E_INVALID
    assert lib.osmodi_source_compressible(plan.handle, u.data_ptr(), u.data_ptr(), 1.0, 0.5, 1.0, 1.0, 1.0,
                                          out.data_ptr(), None, None) == osm.E_INVALID  # gamma must exceed 1
