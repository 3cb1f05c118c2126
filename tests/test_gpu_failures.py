"""Failure statuses, reached without a GPU fault: a grid barrier of the
batched persistent kernel that runs out of polls (OSMODI_E_TIMEOUT), and a
refinement whose residual grows (OSMODI_E_DIVERGED).  Both are driven by the
library's test knobs (osmodi_debug_set); every wait stays bounded, and each
test then solves again to show the GPU and the context still answer."""
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


@pytest.fixture
def knobs(osm):
    yield osm
    for k in (osm.DEBUG_BARRIER_SPINS, osm.DEBUG_SKIP_BARRIER_BLOCK, osm.DEBUG_CORRECTION_SCALE):
        osm.debug_set(k, osm.DEBUG_DEFAULT)


def _rel(a, b, valid):
    return float(np.linalg.norm(a[valid] - b[valid]) / np.linalg.norm(b[valid]))


def _batch(osm, n=4, size=64):
    probs = [inputs.lamb_oseen_2d(n=size, seed=s) for s in range(n)]
    masks = [inputs.random_mask((size, size), p_missing=0.05, seed=s) for s in range(n)]
    plans = [osm.Plan(2, (size, size), pr.spacing, m.cuda()) for pr, m in zip(probs, masks)]
    grads = [pr.grad.cuda() for pr in probs]
    return probs, masks, plans, grads


def test_batched_barrier_time_out_is_reported(knobs):
    osm = knobs
    probs, masks, plans, grads = _batch(osm)
    batch = osm.Batch(plans)
    ps = [torch.zeros((64, 64), dtype=torch.float64, device="cuda") for _ in plans]
    assert osm.debug_set(osm.DEBUG_BARRIER_SPINS, 4096) == 0
    assert osm.debug_set(osm.DEBUG_SKIP_BARRIER_BLOCK, 0) == -1
    st, res = batch.solve(grads, ps, 1e-10, check=False)
    torch.cuda.synchronize()
    assert st == osm.E_TIMEOUT
    # knobs back to their defaults: the same batch solves, to the oracle's answer
    osm.debug_set(osm.DEBUG_BARRIER_SPINS, osm.DEBUG_DEFAULT)
    osm.debug_set(osm.DEBUG_SKIP_BARRIER_BLOCK, osm.DEBUG_DEFAULT)
    for p in ps:
        p.zero_()
    st, res = batch.solve(grads, ps, 1e-10)
    assert st == osm.OK
    for pr, m, p in zip(probs, masks, ps):
        valid = m.numpy().astype(bool)
        want = oracle.solve_direct(oracle.Grid(valid, pr.spacing), pr.grad.numpy())
        assert _rel(p.cpu().numpy(), want, valid) < 1e-8


@pytest.mark.parametrize("precond", [0, 1])
def test_growing_residual_is_reported_as_diverged(knobs, precond):
    osm = knobs
    prob = inputs.sincos_3d(n=24, mask_radius=1.0)
    valid = prob.mask.numpy().astype(bool)
    plan = osm.Plan(3, (24, 24, 24), prob.spacing, prob.mask.cuda(), precision=osm.FP32_REFINE, precond=precond)
    g = prob.grad.cuda()
    p = torch.zeros((24, 24, 24), dtype=torch.float64, device="cuda")
    osm.debug_set(osm.DEBUG_CORRECTION_SCALE, -1000000)
    res = plan.solve(g, p, 1e-11, check=False)
    assert res.status == osm.E_DIVERGED
    osm.debug_set(osm.DEBUG_CORRECTION_SCALE, osm.DEBUG_DEFAULT)
    p.zero_()
    res = plan.solve(g, p, 1e-11)
    assert res.status == osm.OK
    want = oracle.solve_direct(oracle.Grid(valid, prob.spacing), prob.grad.double().numpy())
    assert _rel(p.cpu().numpy(), want, valid) < 1e-9
    plan.close()
