"""The batched persistent solve with the multigrid preconditioner inside the
one launch (plans built with precond = 1), against the oracle, against
single solves and against the plain-CG batch.  Needs a GPU."""
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


def _instances(shapes, seed, ndim=2, hole=0.3):
    """Random masks (a fraction up to `hole` of the cells missing, so some
    instances fall apart into several components) and random gradients."""
    rng = np.random.default_rng(seed)
    out = []
    for i, shape in enumerate(shapes):
        if ndim == 2:
            spacing = (float(rng.uniform(0.05, 0.2)), float(rng.uniform(0.05, 0.2)))
        else:
            spacing = (1.0, 1.0, 1.0) if i % 2 else (1.0, 1.3, 0.7)
        valid = rng.random(shape) > rng.uniform(0.0, hole)
        if not valid.any():
            valid.flat[0] = True
        f = rng.normal(size=(ndim,) + tuple(shape))
        out.append((valid, spacing, f))
    return out


def _plans(osm, inst, ndim=2, precond=1, precision=2):
    plans = []
    for valid, spacing, f in inst:
        m = torch.from_numpy(valid.astype(np.uint8)).cuda()
        plans.append(osm.Plan(ndim, valid.shape[::-1], spacing, m, precond=precond, precision=precision))
    return plans


# (ny, nx): tiny ones without a hierarchy (8 cells or fewer per axis), ones
# whose first coarse level is already small (solved inside one block), and
# ones with two or three grid-wide levels above the in-block ones
SHAPES_2D = [(5, 7), (8, 8), (9, 17), (33, 40), (64, 70), (130, 90), (160, 200), (300, 290), (257, 515), (12, 400)]


@pytest.mark.parametrize("precision", [2, 0])
def test_batched_multigrid_matches_oracle_2d(osm, precision):
    inst = _instances(SHAPES_2D, 11)
    plans = _plans(osm, inst, precision=precision)
    grads = [torch.from_numpy(f).cuda() for _, _, f in inst]
    ps = [torch.zeros(v.shape, dtype=torch.float64, device="cuda") for v, _, _ in inst]
    st, res = osm.Batch(plans).solve(grads, ps, 1e-12)
    assert st == osm.OK, [r.as_dict() for r in res]
    for (valid, spacing, f), p, r in zip(inst, ps, res):
        want = oracle.solve_direct(oracle.Grid(valid, spacing), f)
        got = p.cpu().numpy()
        assert r.status == osm.OK and r.eps_R <= 1e-12
        assert _rel(got, want, valid) < 1e-10
        assert np.isnan(got[~valid]).all()
        assert r.kernel_launches == 1.0


def test_batched_multigrid_needs_few_iterations(osm):
    """The V-cycle inside the launch does what the preconditioner does in a
    single solve: a few dozen iterations where plain CG needs hundreds, and
    about as many as the multigrid single solve of the same instance."""
    probs = [inputs.piv_snapshot_2d(i, size_range=((128, 400), (128, 300))) for i in range(8)]
    out = {}
    for precond in (0, 1):
        plans = [osm.Plan(2, pr.dims, pr.spacing, pr.mask.cuda(), precond=precond) for pr in probs]
        grads = [pr.grad.cuda() for pr in probs]
        ps = [torch.zeros(pr.mask.shape, dtype=torch.float64, device="cuda") for pr in probs]
        st, res = osm.Batch(plans).solve(grads, ps, 1e-10)
        assert st == osm.OK
        out[precond] = ([r.inner_iters for r in res], [p.cpu().numpy() for p in ps])
        if precond == 1:
            single = []
            for pl, pr in zip(plans, probs):
                p1 = torch.zeros(pr.mask.shape, dtype=torch.float64, device="cuda")
                r1 = pl.solve(pr.grad.cuda(), p1, 1e-10)
                single.append(r1.inner_iters)
            out["single"] = single
    it_plain, p_plain = out[0]
    it_mg, p_mg = out[1]
    assert max(it_mg) < 60, it_mg
    assert np.mean(it_mg) * 5 < np.mean(it_plain), (it_mg, it_plain)
    assert np.mean(it_mg) <= 1.5 * np.mean(out["single"]) + 4, (it_mg, out["single"])
    for pr, a, b in zip(probs, p_plain, p_mg):
        valid = pr.mask.numpy().astype(bool)
        assert _rel(b, a, valid) < 1e-8


def test_batched_multigrid_equals_single_solves(osm):
    inst = _instances([(40, 50), (100, 130), (200, 180), (7, 300)], 12)
    plans = _plans(osm, inst)
    singles = []
    for pl, (valid, spacing, f) in zip(plans, inst):
        p1 = torch.zeros(valid.shape, dtype=torch.float64, device="cuda")
        r1 = pl.solve(torch.from_numpy(f).float().cuda(), p1, 1e-11)
        assert r1.status == osm.OK
        singles.append(p1.cpu().numpy())
    grads = [torch.from_numpy(f).float().cuda() for _, _, f in inst]
    ps = [torch.zeros(v.shape, dtype=torch.float64, device="cuda") for v, _, _ in inst]
    st, res = osm.Batch(plans).solve(grads, ps, 1e-11)
    assert st == osm.OK
    for (valid, _, _), p, s in zip(inst, ps, singles):
        assert _rel(p.cpu().numpy(), s, valid) < 1e-9


def test_batched_multigrid_3d(osm):
    rng = np.random.default_rng(13)
    shapes = [tuple(int(v) for v in rng.integers(5, 30, size=3)) for _ in range(6)] + [(33, 34, 35)]
    inst = _instances(shapes, 14, ndim=3, hole=0.2)
    plans = _plans(osm, inst, ndim=3)
    grads = [torch.from_numpy(f).cuda() for _, _, f in inst]
    ps = [torch.zeros(v.shape, dtype=torch.float64, device="cuda") for v, _, _ in inst]
    st, res = osm.Batch(plans).solve(grads, ps, 1e-11)
    assert st == osm.OK, [r.as_dict() for r in res]
    for (valid, spacing, f), p, r in zip(inst, ps, res):
        want = oracle.solve_direct(oracle.Grid(valid, spacing), f)
        assert _rel(p.cpu().numpy(), want, valid) < 1e-9
        assert r.inner_iters < 80


def test_batched_multigrid_graph_replays(osm):
    """The multigrid batch captured as one graph: replays with new gradients
    give the oracle's answers and the direct launch's iteration counts."""
    inst = _instances([(30, 41), (90, 77), (150, 260), (6, 6)], 15)
    plans = _plans(osm, inst)
    grads = [torch.from_numpy(f).float().cuda() for _, _, f in inst]
    ps = [torch.zeros(v.shape, dtype=torch.float64, device="cuda") for v, _, _ in inst]
    batch = osm.Batch(plans)
    graph = batch.capture(grads, ps, 1e-11)
    rng = np.random.default_rng(78)
    for rep in range(2):
        fields = [f if rep == 0 else rng.normal(size=f.shape) for (_, _, f) in inst]
        for g, f, p in zip(grads, fields, ps):
            g.copy_(torch.from_numpy(f).float())
            p.zero_()
        graph.launch()
        st, res = graph.results()
        assert st == osm.OK
        got = [p.cpu().numpy() for p in ps]
        for (valid, spacing, _), f, g_np in zip(inst, fields, got):
            want = oracle.solve_direct(oracle.Grid(valid, spacing), np.asarray(f, np.float32).astype(np.float64))
            assert _rel(g_np, want, valid) < 1e-9
        direct = [torch.zeros_like(p) for p in ps]
        st2, res2 = batch.solve(grads, direct, 1e-11)
        assert st2 == osm.OK
        for (valid, _, _), a, b, r1, r2 in zip(inst, got, direct, res, res2):
            assert r1.inner_iters == r2.inner_iters
            assert _rel(a, b.cpu().numpy(), valid) < 1e-12
    graph.close()


def test_batched_multigrid_isolates_bad_input_and_zero_field(osm):
    inst = _instances([(50, 60), (120, 140), (80, 80)], 16)
    inst[2] = (inst[2][0], inst[2][1], np.zeros_like(inst[2][2]))
    plans = _plans(osm, inst)
    grads = [torch.from_numpy(f).float().cuda() for _, _, f in inst]
    ps = [torch.zeros(v.shape, dtype=torch.float64, device="cuda") for v, _, _ in inst]
    v0 = inst[0][0]
    j, i = np.argwhere(v0)[0]
    grads[0][1, j, i] = float("nan")
    ps[0].fill_(2.0)
    st, res = osm.Batch(plans).solve(grads, ps, 1e-11)
    assert st == osm.E_NAN_INPUT
    assert res[0].status == osm.E_NAN_INPUT and (ps[0].cpu().numpy() == 2.0).all()
    assert res[2].status == osm.OK and res[2].inner_iters == 0
    valid, spacing, f = inst[1]
    want = oracle.solve_direct(oracle.Grid(valid, spacing), np.asarray(f, np.float32).astype(np.float64))
    assert res[1].status == osm.OK and _rel(ps[1].cpu().numpy(), want, valid) < 1e-9


def test_batched_multigrid_split_does_not_change_the_cycle(osm):
    """Which coarse levels run grid-wide and which inside one block per
    instance changes where the V-cycle runs, not what it computes: the same
    iterations and the same answers for every split."""
    probs = [inputs.piv_snapshot_2d(i, size_range=((200, 700), (150, 400))) for i in range(6)]
    plans = [osm.Plan(2, pr.dims, pr.spacing, pr.mask.cuda(), precond=1) for pr in probs]
    grads = [pr.grad.cuda() for pr in probs]
    runs = []
    try:
        for bottom in (0, 1 << 30, 300, 16):
            osm.debug_set(osm.DEBUG_BATCH_BOTTOM_CELLS, bottom)
            ps = [torch.zeros(pr.mask.shape, dtype=torch.float64, device="cuda") for pr in probs]
            st, res = osm.Batch(plans).solve(grads, ps, 1e-10)
            assert st == osm.OK
            runs.append(([r.inner_iters for r in res], [p.cpu().numpy() for p in ps]))
    finally:
        osm.debug_set(osm.DEBUG_BATCH_BOTTOM_CELLS, osm.DEBUG_DEFAULT)
    its0, p0 = runs[0]
    assert max(its0) < 30, its0
    for its, ps in runs[1:]:
        assert its == its0
        for pr, a, b in zip(probs, ps, p0):
            valid = pr.mask.numpy().astype(bool)
            assert _rel(a, b, valid) < 1e-12
