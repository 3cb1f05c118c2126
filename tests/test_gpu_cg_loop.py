"""The captured CG as one graph with a device-side loop (a conditional while
node that stops at convergence) against graphs of check_every iterations
relaunched by the host: the same kernels in the same order, so the same
iterations and the same result bit for bit, with fewer kernels launched.
Needs a GPU."""
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


def _run(osm, plan, grad, fixed, tol):
    old = osm.debug_set(osm.DEBUG_CG_FIXED_GRAPH, 1 if fixed else 0)
    try:
        p = torch.zeros(grad.shape[1:], dtype=torch.float64, device="cuda")
        res = plan.solve(grad, p, tol)
    finally:
        osm.debug_set(osm.DEBUG_CG_FIXED_GRAPH, old)
    return res, p.cpu().numpy()


@pytest.mark.parametrize("ndim,precond,precision", [(3, 1, 2), (3, 1, 0), (2, 0, 2), (2, 1, 2)])
def test_loop_graph_equals_fixed_chunks(osm, ndim, precond, precision):
    if ndim == 3:
        n = 72
        prob = inputs.gaussian_blobs_3d(n=(n, n, n), n_blobs=6)
        mask = inputs.random_mask((n, n, n), p_missing=0.03, seed=21)
        dims, spacing = (n, n, n), (1.0, 1.0, 1.0)
    else:
        prob = inputs.piv_snapshot_2d(3, size_range=((200, 300), (150, 250)))
        mask, dims, spacing = prob.mask, prob.dims, prob.spacing
    grad = prob.grad.cuda()
    if precision == 0:
        grad = grad.double()
    plan = osm.Plan(ndim, dims, spacing, mask.cuda(), precond=precond, precision=precision)
    r_loop, p_loop = _run(osm, plan, grad, False, 1e-10)
    r_fix, p_fix = _run(osm, plan, grad, True, 1e-10)
    r_loop2, p_loop2 = _run(osm, plan, grad, False, 1e-10)  # the cached loop graph, relaunched
    plan.close()
    for r in (r_loop, r_fix, r_loop2):
        assert r.status == osm.OK and r.eps_R <= 1e-10, r.as_dict()
    assert r_loop.inner_iters == r_fix.inner_iters == r_loop2.inner_iters
    valid = mask.numpy().astype(bool)
    assert np.array_equal(p_loop[valid], p_fix[valid]) and np.array_equal(p_loop2[valid], p_loop[valid])
    assert r_loop.kernel_launches < r_fix.kernel_launches, (r_loop.kernel_launches, r_fix.kernel_launches)
    want = oracle.solve_direct(oracle.Grid(valid, spacing), grad.double().cpu().numpy()) if ndim == 2 else None
    if want is not None:
        assert np.linalg.norm(p_loop[valid] - want[valid]) <= 1e-8 * np.linalg.norm(want[valid])


def test_loop_graph_runs_past_its_cap(osm):
    """Plain CG on a large 2-D field takes far more iterations than one graph
    launch's loop cap (64 bodies of two): the host relaunches the graph until
    the device reports convergence, with the fixed chunks' answer."""
    prob = inputs.piv_snapshot_2d(5, size_range=((500, 600), (400, 500)))
    plan = osm.Plan(2, prob.dims, prob.spacing, prob.mask.cuda(), precond=0)
    grad = prob.grad.cuda()
    r_loop, p_loop = _run(osm, plan, grad, False, 1e-10)
    r_fix, p_fix = _run(osm, plan, grad, True, 1e-10)
    plan.close()
    assert r_loop.status == osm.OK and r_fix.status == osm.OK
    assert r_loop.inner_iters == r_fix.inner_iters and r_loop.inner_iters > 128, r_loop.inner_iters
    valid = prob.mask.numpy().astype(bool)
    assert np.array_equal(p_loop[valid], p_fix[valid])
