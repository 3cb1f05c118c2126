"""The batched persistent solve against the oracle and against single
solves.  Needs a GPU."""
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


def _random_instances(n, seed, ndim=2):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        if ndim == 2:
            shape = (int(rng.integers(3, 70)), int(rng.integers(5, 90)))
            spacing = (float(rng.uniform(0.05, 0.2)), float(rng.uniform(0.05, 0.2)))
        else:
            shape = tuple(int(v) for v in rng.integers(3, 14, size=3))
            spacing = (1.0, 1.0, 1.0) if i % 2 else (1.0, 1.3, 0.7)
        valid = rng.random(shape) > rng.uniform(0.0, 0.3)
        if not valid.any():
            valid.flat[0] = True
        f = rng.normal(size=(ndim,) + shape)
        out.append((valid, spacing, f))
    return out


@pytest.mark.parametrize("precision", [2, 0])
def test_batched_matches_oracle_2d(osm, precision):
    inst = _random_instances(14, 1)
    plans, grads, ps = [], [], []
    for valid, spacing, f in inst:
        plans.append(osm.Plan(2, valid.shape[::-1], spacing, torch.from_numpy(valid.astype(np.uint8)).cuda(),
                              precision=precision))
        grads.append(torch.from_numpy(f).cuda())
        ps.append(torch.zeros(valid.shape, dtype=torch.float64, device="cuda"))
    st, res = osm.Batch(plans).solve(grads, ps, 1e-12)
    assert st == osm.OK, [r.as_dict() for r in res]
    for (valid, spacing, f), p, r in zip(inst, ps, res):
        want = oracle.solve_direct(oracle.Grid(valid, spacing), f)
        got = p.cpu().numpy()
        assert r.status == osm.OK and r.eps_R <= 1e-12
        assert _rel(got, want, valid) < 1e-10
        assert np.isnan(got[~valid]).all()


def test_batched_equals_single_solves_and_isolates_bad_input(osm):
    inst = _random_instances(9, 2)
    plans, grads, ps, singles = [], [], [], []
    for k, (valid, spacing, f) in enumerate(inst):
        m = torch.from_numpy(valid.astype(np.uint8)).cuda()
        plan = osm.Plan(2, valid.shape[::-1], spacing, m)
        g = torch.from_numpy(f).float().cuda()
        p1 = torch.zeros(valid.shape, dtype=torch.float64, device="cuda")
        plan.solve(g, p1, 1e-11)
        singles.append(p1.cpu().numpy())
        plans.append(plan)
        grads.append(g)
        ps.append(torch.zeros(valid.shape, dtype=torch.float64, device="cuda"))
    # instance 4 gets a NaN at a valid cell: it alone fails, untouched
    bad = 4
    vb = inst[bad][0]
    j, i = np.argwhere(vb)[0]
    grads[bad][0, j, i] = float("nan")
    ps[bad].fill_(3.0)
    st, res = osm.Batch(plans).solve(grads, ps, 1e-11)
    assert st == osm.E_NAN_INPUT
    for k, ((valid, spacing, f), p, r) in enumerate(zip(inst, ps, res)):
        got = p.cpu().numpy()
        if k == bad:
            assert r.status == osm.E_NAN_INPUT and (got == 3.0).all()
        else:
            assert r.status == osm.OK
            assert _rel(got, singles[k], valid) < 1e-9


def test_batched_piv_snapshots(osm):
    """Snapshots of the PIV-like workload (elliptical solid masks, FP32
    gradients), reduced sizes so the oracle finishes quickly."""
    probs = [inputs.piv_snapshot_2d(i, size_range=((64, 160), (64, 120))) for i in range(10)]
    plans, grads, ps = [], [], []
    for pr in probs:
        plans.append(osm.Plan(2, pr.dims, pr.spacing, pr.mask.cuda()))
        grads.append(pr.grad.cuda())
        ps.append(torch.zeros(pr.mask.shape, dtype=torch.float64, device="cuda"))
    st, res = osm.Batch(plans).solve(grads, ps, 1e-11)
    assert st == osm.OK
    for pr, p, r in zip(probs, ps, res):
        valid = pr.mask.numpy().astype(bool)
        grid = oracle.Grid(valid, pr.spacing)
        want, it, e = oracle.solve_cg(grid, pr.grad.double().numpy(), tol=1e-14, maxit=40000)
        assert _rel(p.cpu().numpy(), want, valid) < 1e-9


def test_batched_3d(osm):
    inst = _random_instances(6, 3, ndim=3)
    plans, grads, ps = [], [], []
    for valid, spacing, f in inst:
        plans.append(osm.Plan(3, valid.shape[::-1], spacing, torch.from_numpy(valid.astype(np.uint8)).cuda()))
        grads.append(torch.from_numpy(f).cuda())
        ps.append(torch.zeros(valid.shape, dtype=torch.float32, device="cuda"))
    st, res = osm.Batch(plans).solve(grads, ps, 1e-10)
    assert st == osm.OK
    for (valid, spacing, f), p in zip(inst, ps):
        want = oracle.solve_direct(oracle.Grid(valid, spacing), f)
        assert _rel(p.cpu().numpy().astype(np.float64), want, valid) < 1e-6


def test_batched_zero_gradient_and_repeat(osm):
    """An instance with S = 0 finishes at once while the others continue;
    repeating the call on the same workspace gives the same answer (to
    rounding: instances with several connected components add their
    per-component means with atomics, whose order varies)."""
    inst = _random_instances(5, 4)
    inst[2] = (inst[2][0], inst[2][1], np.zeros_like(inst[2][2]))
    plans = [osm.Plan(2, v.shape[::-1], s, torch.from_numpy(v.astype(np.uint8)).cuda()) for v, s, f in inst]
    batch = osm.Batch(plans)
    outs = []
    for rep in range(2):
        grads = [torch.from_numpy(f).cuda() for v, s, f in inst]
        ps = [torch.zeros(v.shape, dtype=torch.float64, device="cuda") for v, s, f in inst]
        st, res = batch.solve(grads, ps, 1e-11)
        assert st == osm.OK
        assert res[2].inner_iters == 0 and res[2].eps_R == 0.0
        outs.append([p.cpu().numpy() for p in ps])
    for a, b, (v, s, f) in zip(outs[0], outs[1], inst):
        np.testing.assert_allclose(a[v], b[v], rtol=1e-12, atol=1e-14)


def test_batched_autotune_tile_depth(osm):
    inst = _random_instances(7, 6)
    plans = [osm.Plan(2, v.shape[::-1], s, torch.from_numpy(v.astype(np.uint8)).cuda()) for v, s, f in inst]
    batch = osm.Batch(plans)
    grads = [torch.from_numpy(f).cuda() for v, s, f in inst]
    ps = [torch.zeros(v.shape, dtype=torch.float64, device="cuda") for v, s, f in inst]
    depth = batch.autotune(grads, ps)
    assert depth in (1, 2, 4, 8)
    for p in ps:
        p.zero_()
    st, res = batch.solve(grads, ps, 1e-11)
    assert st == osm.OK
    for (valid, spacing, f), p in zip(inst, ps):
        want = oracle.solve_direct(oracle.Grid(valid, spacing), f)
        assert _rel(p.cpu().numpy(), want, valid) < 1e-9


def test_captured_graph_replays_new_gradients(osm):
    """The batch captured as a CUDA graph: each replay with new gradients
    written into the bound buffers gives the oracle's answer for those
    gradients, and agrees with the direct batched solve."""
    inst = _random_instances(10, 5)
    plans, grads, ps = [], [], []
    for valid, spacing, f in inst:
        plans.append(osm.Plan(2, valid.shape[::-1], spacing, torch.from_numpy(valid.astype(np.uint8)).cuda()))
        grads.append(torch.from_numpy(f).float().cuda())
        ps.append(torch.zeros(valid.shape, dtype=torch.float64, device="cuda"))
    batch = osm.Batch(plans)
    graph = batch.capture(grads, ps, 1e-12)
    rng = np.random.default_rng(77)
    for rep in range(3):
        fields = [f if rep == 0 else rng.normal(size=f.shape) for (_, _, f) in inst]
        for g, f, p in zip(grads, fields, ps):
            g.copy_(torch.from_numpy(f).float())
            p.zero_()
        graph.launch()
        st, res = graph.results()
        assert st == osm.OK, [r.as_dict() for r in res]
        got = [p.cpu().numpy() for p in ps]
        for (valid, spacing, _), f, g_np, r in zip(inst, fields, got, res):
            want = oracle.solve_direct(oracle.Grid(valid, spacing), np.asarray(f, np.float32).astype(np.float64))
            assert r.status == osm.OK and r.eps_R <= 1e-12 and r.ms > 0
            assert _rel(g_np, want, valid) < 1e-9
        # the direct launch of the same batch lands on the same answers
        direct = [torch.zeros_like(p) for p in ps]
        st2, res2 = batch.solve(grads, direct, 1e-12)
        assert st2 == osm.OK
        for (valid, _, _), a, b, r1, r2 in zip(inst, got, direct, res, res2):
            assert r1.inner_iters == r2.inner_iters
            assert _rel(a, b.cpu().numpy(), valid) < 1e-12
    graph.close()


@pytest.mark.parametrize("precond", [0, 1])
def test_solve_many_streams_match_oracle(osm, precond):
    """osmodi_solve_many: the single-problem solve of every plan spread over
    four streams and host threads; each answer equals the oracle's and the
    per-plan result of a plain osmodi_solve."""
    inst = _random_instances(11, 9)
    plans, grads, ps = [], [], []
    for valid, spacing, f in inst:
        plans.append(osm.Plan(2, valid.shape[::-1], spacing, torch.from_numpy(valid.astype(np.uint8)).cuda(),
                              precond=precond))
        grads.append(torch.from_numpy(f).float().cuda())
        ps.append(torch.zeros(valid.shape, dtype=torch.float64, device="cuda"))
    many = osm.Many(plans, streams=4)
    for rep in range(2):  # the second pass replays every plan's captured graphs
        for p in ps:
            p.zero_()
        st, res = many.solve(grads, ps, 1e-12)
        assert st == osm.OK, [r.as_dict() for r in res]
        for (valid, spacing, f), p, r in zip(inst, ps, res):
            want = oracle.solve_direct(oracle.Grid(valid, spacing), np.asarray(f, np.float32).astype(np.float64))
            assert r.status == osm.OK and r.eps_R <= 1e-12 and r.kernel_launches > 0
            assert _rel(p.cpu().numpy(), want, valid) < 1e-9
    # same iterations as one-by-one solves
    for k in (0, 5, 10):
        p1 = torch.zeros_like(ps[k])
        r1 = plans[k].solve(grads[k], p1, 1e-12)
        assert r1.inner_iters == res[k].inner_iters


def test_solve_many_rejects_a_plan_shared_across_streams(osm):
    """A plan carries per-solve host state: listed twice, it must map to one
    stream (indices congruent mod the stream count), else nothing runs."""
    inst = _random_instances(3, 4)
    plans = [osm.Plan(2, v.shape[::-1], sp, torch.from_numpy(v.astype(np.uint8)).cuda()) for v, sp, _ in inst]
    grads = [torch.from_numpy(f).float().cuda() for _, _, f in inst]

    def buffers(order):  # each problem's gradient and a pressure of its plan's shape
        return ([grads[k] for k in order],
                [torch.zeros(inst[k][0].shape, dtype=torch.float64, device="cuda") for k in order])

    # plans[0] at indices 0 and 1 on two streams: rejected
    g_bad, p_bad = buffers([0, 0, 1])
    st, _ = osm.Many([plans[0], plans[0], plans[1]], streams=2).solve(g_bad, p_bad, 1e-10, check=False)
    assert st == osm.E_INVALID
    # plans[0] at indices 0 and 2 on two streams (both on stream 0): solved in turn
    g_ok, p_ok = buffers([0, 1, 0])
    st, res = osm.Many([plans[0], plans[1], plans[0]], streams=2).solve(g_ok, p_ok, 1e-10)
    assert st == osm.OK and all(r.status == osm.OK for r in res)
    # the same problem solved twice in turn: the same answer (missing cells
    # NaN in both; per-component sums use atomic adds, so the last bits may
    # differ)
    torch.testing.assert_close(p_ok[0], p_ok[2], rtol=1e-12, atol=1e-14, equal_nan=True)
