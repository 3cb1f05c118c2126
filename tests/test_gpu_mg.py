"""The multigrid-preconditioned CG solve (osmodi_options.precond = 1)
against the oracle: the same fixed point to the same tolerance as plain CG,
in far fewer iterations, on every grid shape the hierarchy meets (ragged
sizes, masks with several components, one-cell-thick axes, grids too small
for a coarse level).  Needs a GPU."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_16935_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osm():
    from paper_2311_16935_gb300 import build

    build.build()
    from paper_2311_16935_gb300 import osmodi

    return osmodi


def _rel(a, b, valid):
    return float(np.linalg.norm(a[valid] - b[valid]) / max(np.linalg.norm(b[valid]), 1e-300))


def _solve(osm, f, valid, spacing, tol, **opt):
    plan = osm.Plan(valid.ndim, valid.shape[::-1], spacing, torch.from_numpy(valid.astype(np.uint8)).cuda(), **opt)
    p = torch.zeros(valid.shape, dtype=torch.float64, device="cuda")
    res = plan.solve(torch.from_numpy(np.ascontiguousarray(f)).cuda(), p, tol)
    return plan, res, p.cpu().numpy()


SHAPES = [((37, 53), (0.1, 0.13)), ((130, 9), (1.0, 1.0)), ((19, 23, 29), (1.0, 1.0, 1.0)),
          ((17, 1, 33), (1.0, 1.0, 1.0)), ((9, 12, 40), (1.0, 1.3, 0.7))]


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("case", range(len(SHAPES)))
def test_preconditioned_matches_oracle(osm, case, precision):
    shape, spacing = SHAPES[case]
    rng = np.random.default_rng(60 + case)
    valid = rng.random(shape) > 0.2  # salt-and-pepper: several components
    f = rng.normal(size=(len(shape),) + shape)
    if precision == 2:
        f = f.astype(np.float32)
    want = oracle.solve_direct(oracle.Grid(valid, spacing), f.astype(np.float64))
    _, r0, p0 = _solve(osm, f, valid, spacing, 1e-12, precision=precision)
    _, r1, p1 = _solve(osm, f, valid, spacing, 1e-12, precision=precision, precond=1)
    assert r0.status == osm.OK and r1.status == osm.OK, (r0.as_dict(), r1.as_dict())
    assert r1.eps_R <= 1e-12
    assert _rel(p1, want, valid) < 1e-10
    assert np.isnan(p1[~valid]).all()
    assert r1.inner_iters < r0.inner_iters, (r1.inner_iters, r0.inner_iters)


def test_preconditioned_configs_and_iteration_counts(osm):
    """The 64^2 Lamb-Oseen and 128^3 sin-cos configurations to 1e-10 against
    the oracle, each in a small fraction of plain CG's iterations."""
    prob = inputs.lamb_oseen_2d(n=64)
    valid = prob.mask.numpy().astype(bool)
    f = prob.grad.numpy()
    want = oracle.solve_direct(oracle.Grid(valid, prob.spacing), f)
    _, r0, _ = _solve(osm, f, valid, prob.spacing, 1e-10, precision=0)
    _, r1, got = _solve(osm, f, valid, prob.spacing, 1e-10, precision=0, precond=1)
    assert r1.status == osm.OK and _rel(got, want, valid) < 1e-9
    assert r1.inner_iters * 3 < r0.inner_iters, (r1.inner_iters, r0.inner_iters)

    prob = inputs.sincos_3d(n=128)
    valid = prob.mask.numpy().astype(bool)
    f = prob.grad.numpy()
    _, r0, _ = _solve(osm, f, valid, prob.spacing, 1e-12)
    _, r1, got = _solve(osm, f, valid, prob.spacing, 1e-12, precond=1)
    assert r1.status == osm.OK
    want = oracle.solve_cg(oracle.Grid(valid, prob.spacing), f.astype(np.float64), tol=1e-14, maxit=20000)[0]
    assert _rel(got, want, valid) < 1e-10
    assert r1.inner_iters * 8 < r0.inner_iters, (r1.inner_iters, r0.inner_iters)


def test_preconditioned_small_grid_and_noalloc(osm):
    """A grid of at most 8 cells per axis has no coarse level (plain CG); the
    allocation-free entry runs the preconditioned solve too."""
    rng = np.random.default_rng(3)
    valid = rng.random((6, 8)) > 0.2
    f = rng.normal(size=(2, 6, 8))
    want = oracle.solve_direct(oracle.Grid(valid, (1.0, 1.0)), f)
    _, r, got = _solve(osm, f, valid, (1.0, 1.0), 1e-12, precision=0, precond=1)
    assert r.status == osm.OK and _rel(got, want, valid) < 1e-10
    valid = rng.random((40, 50)) > 0.1
    f = rng.normal(size=(2, 40, 50))
    want = oracle.solve_direct(oracle.Grid(valid, (1.0, 1.0)), f)
    plan = osm.Plan(2, (50, 40), (1.0, 1.0), torch.from_numpy(valid.astype(np.uint8)).cuda(), precond=1)
    p = torch.zeros((40, 50), dtype=torch.float64, device="cuda")
    res = plan.solve_noalloc(torch.from_numpy(f).cuda(), p, 1e-12)
    assert res.status == osm.OK and _rel(p.cpu().numpy(), want, valid) < 1e-10


def test_preconditioner_timing_is_reported(osm):
    prob = inputs.sincos_3d(n=48)
    valid = prob.mask.numpy().astype(bool)
    plan, res, _ = _solve(osm, prob.grad.numpy(), valid, prob.spacing, 1e-10, precond=1, profile=1)
    ks = plan.kernel_stats()
    assert res.status == osm.OK
    assert ks["precond_applications"] > 0 and ks["precond_ms"] > 0
    assert ks["precond_applications"] <= ks["cg_update_launches"]


@pytest.mark.parametrize("sweeps,scale", [(1, 1.8), (3, 2.0), (2, 1.0), (1, 3.5)])
def test_smoothing_options_keep_the_fixed_point(osm, sweeps, scale):
    """options.mg_sweeps / mg_scale change the preconditioner, never the
    answer: any positive scale keeps it symmetric positive definite, so CG
    reaches the oracle's fixed point (3-D red-black and 2-D Jacobi)."""
    for shape, spacing in (((21, 26, 30), (1.0, 1.1, 0.9)), ((45, 61), (0.2, 0.2))):
        rng = np.random.default_rng(7 + sweeps)
        valid = rng.random(shape) > 0.15
        f = rng.normal(size=(len(shape),) + shape)
        want = oracle.solve_direct(oracle.Grid(valid, spacing), f)
        _, res, got = _solve(osm, f, valid, spacing, 1e-12, precision=0, precond=1, mg_sweeps=sweeps,
                             mg_scale=scale)
        assert res.status == osm.OK, res.as_dict()
        assert _rel(got, want, valid) < 1e-10


@pytest.mark.parametrize("shape", [(19, 23, 29), (33, 30, 61), (5, 40, 17), (64, 64, 64), (21, 37, 300)])
def test_fused_sweeps_equal_half_sweeps(osm, shape):
    """The fused one-pass red-black sweeps (default; with the fine level's
    inputs staged by TMA; with them loaded a plane ahead; staged by
    cp.async) against the same
    V-cycle by one-colour
    half-sweeps on every level (OSMODI_DEBUG_MG_UNFUSED): the same arithmetic,
    so the preconditioned CG takes the same iterations, reports the same
    residual (to FP32 rounding of the preconditioner) and lands on the same
    answer.  The shapes cover several tiles and slabs with ragged edges in
    every axis, a mask with several components and FP32 inner sweeps."""
    rng = np.random.default_rng(sum(shape))
    valid = rng.random(shape) > 0.15
    f = rng.normal(size=(3,) + shape).astype(np.float32)
    spacing = (1.0, 1.0, 1.0)
    out = {}
    for variant in (0, 1, 2, 3, 4):  # fused, half-sweeps, TMA-staged, prefetching, cp.async-staged
        osm.debug_set(osm.DEBUG_MG_UNFUSED, variant)
        try:
            _, res, p = _solve(osm, f, valid, spacing, 1e-11, precision=2, precond=1)
        finally:
            osm.debug_set(osm.DEBUG_MG_UNFUSED, osm.DEBUG_DEFAULT)
        assert res.status == osm.OK, res.as_dict()
        out[variant] = (res, p)
    want = oracle.solve_cg(oracle.Grid(valid, spacing), f.astype(np.float64), tol=1e-14, maxit=50000)[0]
    ru, pu = out[1]
    for variant in (0, 2, 3, 4):
        rf, pf = out[variant]
        # rounding (FMA contraction may differ between the kernels) can move a
        # stopping test across its threshold by at most one check chunk
        assert abs(rf.inner_iters - ru.inner_iters) <= 8, (variant, rf.inner_iters, ru.inner_iters)
        assert rf.eps_R <= 1e-11 and ru.eps_R <= 1e-11
        assert _rel(pf, pu, valid) < 1e-10
        assert _rel(pf, want, valid) < 1e-9
