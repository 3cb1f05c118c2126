"""osmodi_solve_noalloc -- the solve for callers that cannot allocate device
memory when they solve (an embedding framework's allocator owns the device
memory, or cudaMalloc/cudaFree would stall a latency-bound loop).  It must
give what osmodi_solve gives, call after call, although its scratch is one
shared device array that keeps the previous call's contents.

Kept in its own file, collected last, so that a run stopping at the first
failure has already run every other test."""
import ctypes
import gc

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


def test_noalloc_switches_plans_and_warm_starts(osm):
    """Two plans of different dimension and shape take turns on the one shared
    scratch (each call finds the other plan's leftovers there), and warm
    starts from a nonzero initial pressure: every call equals osmodi_solve
    with a workspace, given the same initial pressure."""
    p2 = inputs.lamb_oseen_2d(n=80, seed=4)
    v2 = inputs.random_mask((80, 80), p_missing=0.05, seed=8).numpy().astype(bool)
    p3 = inputs.sincos_3d(n=36, mask_radius=1.5)
    v3 = p3.mask.numpy().astype(bool)
    planA = osm.Plan(2, (80, 80), p2.spacing, torch.from_numpy(v2.astype(np.uint8)).cuda())
    planB = osm.Plan(3, (36, 36, 36), p3.spacing, p3.mask.cuda())
    cases = {"A": (planA, p2.grad.cuda(), v2, (80, 80)), "B": (planB, p3.grad.cuda(), v3, (36, 36, 36))}
    gen = torch.Generator().manual_seed(11)
    for name, warm in (("A", False), ("B", False), ("A", True), ("B", True), ("A", False)):
        plan, g, valid, shape = cases[name]
        p0 = torch.randn(shape, generator=gen, dtype=torch.float64) if warm else torch.zeros(shape, dtype=torch.float64)
        p_ref = p0.cuda()
        r_ref = plan.solve(g, p_ref, 1e-11)
        p_new = p0.cuda()
        st, res = _call_noalloc(osm, plan, g, p_new, 1e-11)
        assert st == osm.OK and r_ref.status == osm.OK, (name, warm, st)
        assert _rel(p_new.cpu().numpy(), p_ref.cpu().numpy(), valid) < 1e-10, (name, warm)
        assert np.isnan(p_new.cpu().numpy()[~valid]).all()
        if warm:  # the seed distance is reported the same way by both calls
            assert res.seed_rel_dist > 0 and abs(res.seed_rel_dist - r_ref.seed_rel_dist) < 1e-6
    planA.close()
    planB.close()


def test_noalloc_allocates_nothing(osm):
    """After plan creation (which loads the scratch on the device) and one
    call that has launched each kernel the solve uses once (under lazy module
    loading the driver may load a kernel's code at its first launch), a call
    leaves the device's free memory and torch's allocator untouched."""
    prob = inputs.sincos_3d(n=32, mask_radius=1.2)
    plan = osm.Plan(3, (32, 32, 32), prob.spacing, prob.mask.cuda())
    g = prob.grad.cuda()
    p = torch.zeros((32, 32, 32), dtype=torch.float64, device="cuda")
    # tensors of earlier tests freed by Python's collector would show up as
    # changes of torch's count: collect first, and not during the window
    gc.collect()
    gc.disable()
    try:
        torch.cuda.synchronize()
        alloc0 = torch.cuda.memory_allocated()
        st, _ = _call_noalloc(osm, plan, g, p, 1e-10)
        torch.cuda.synchronize()
        assert st == osm.OK
        assert torch.cuda.memory_allocated() == alloc0
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            p.zero_()
            st, res = _call_noalloc(osm, plan, g, p, 1e-10)
            torch.cuda.synchronize()
            assert st == osm.OK and res.eps_R <= 1e-10
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_allocated() == alloc0
    finally:
        gc.enable()
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
