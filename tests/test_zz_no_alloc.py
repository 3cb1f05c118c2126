"""osmodi_solve_noalloc -- the solve for callers that cannot allocate device
memory when they solve (an embedding framework's allocator owns the device
memory, or cudaMalloc/cudaFree would stall a latency-bound loop).  It must
give what osmodi_solve gives, call after call, although its scratch is one
shared device array that keeps the previous call's contents.

Kept in its own file, collected last, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2311_16935_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osm():
    from paper_2311_16935_gb300 import build

    build.build()
    from paper_2311_16935_gb300 import osmodi

    assert torch.cuda.is_available()
    return osmodi


def _call_noalloc(osm, plan, grad, p, tol):
    """Straight through the C interface (ctypes), no workspace argument."""
    res = osm.osmodi_result()
    stream = torch.cuda.current_stream().cuda_stream
    st = osm.lib().osmodi_solve_noalloc(plan.handle, ctypes.c_void_p(grad.data_ptr()), osm._dtype_code(grad),
                                        ctypes.c_void_p(p.data_ptr()), osm._dtype_code(p), ctypes.c_double(tol),
                                        ctypes.c_int(1 << 30), ctypes.c_void_p(stream), ctypes.byref(res))
    return st, res


def _rel(a, b, valid):
    return float(np.linalg.norm(a[valid] - b[valid]) / np.linalg.norm(b[valid]))


@pytest.mark.parametrize("precision", [0, 2])
def test_noalloc_matches_workspace_solve_twice(osm, precision):
    n = 96
    valid = inputs.random_mask((n, n), p_missing=0.05, seed=5).numpy().astype(bool)
    mask = torch.from_numpy(valid.astype(np.uint8)).cuda()
    probs = [inputs.lamb_oseen_2d(n=n, seed=s) for s in (1, 2)]
    plan = osm.Plan(2, (n, n), probs[0].spacing, mask, precision=precision)
    assert plan.workspace_bytes() <= 16 * 1024 * 1024
    tol = 1e-11
    for prob in probs:  # two calls in a row, different inputs
        g = prob.grad.cuda()
        p_ref = torch.zeros((n, n), dtype=torch.float64, device="cuda")
        r_ref = plan.solve(g, p_ref, tol)
        p_new = torch.full((n, n), 0.0, dtype=torch.float64, device="cuda")
        st, res = _call_noalloc(osm, plan, g, p_new, tol)
        assert st == osm.OK and r_ref.status == osm.OK
        a, b = p_new.cpu().numpy(), p_ref.cpu().numpy()
        assert _rel(a, b, valid) < 1e-10
        assert np.isnan(a[~valid]).all()
        assert res.eps_R <= tol
    plan.close()


def test_noalloc_3d_and_second_plan(osm):
    """A second plan on the same device reuses the scratch the first left."""
    prob = inputs.sincos_3d(n=40, mask_radius=1.5)
    valid = prob.mask.numpy().astype(bool)
    plan = osm.Plan(3, (40, 40, 40), prob.spacing, prob.mask.cuda())
    g = prob.grad.cuda()
    out = []
    for call in range(2):
        p_ref = torch.zeros((40, 40, 40), dtype=torch.float64, device="cuda")
        plan.solve(g, p_ref, 1e-11)
        p_new = torch.zeros_like(p_ref)
        st, res = _call_noalloc(osm, plan, g, p_new, 1e-11)
        assert st == osm.OK
        assert _rel(p_new.cpu().numpy(), p_ref.cpu().numpy(), valid) < 1e-10
        out.append(p_new.cpu().numpy())
    np.testing.assert_array_equal(out[0][valid], out[1][valid])
    plan.close()


def test_noalloc_rejects_plans_beyond_the_scratch(osm):
    plan = osm.Plan(3, (200, 200, 200), (1.0, 1.0, 1.0), None)
    assert plan.workspace_bytes() > 16 * 1024 * 1024
    g = torch.zeros((3, 1, 1, 1), dtype=torch.float32, device="cuda")  # never read
    p = torch.zeros((1,), dtype=torch.float64, device="cuda")
    st, res = _call_noalloc(osm, plan, g, p, 1e-8)
    assert st == osm.E_WORKSPACE
    assert "OSMODI_NOALLOC_SCRATCH_BYTES" in osm.last_cuda_error()
    plan.close()
