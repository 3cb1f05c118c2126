"""The seed network's GPU kernels against the CPU reference (forward and
parameter gradients, BF16 tolerance), and what the trained network gains the
solve.  Needs a GPU."""
import numpy as np
import pytest
import torch

from oracle import net as onet
from paper_2311_16935_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def osm():
    from paper_2311_16935_gb300 import build

    build.build()
    from paper_2311_16935_gb300 import osmodi

    return osmodi


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _problem(n, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    valid = ((x - n / 2) ** 2 + (y - n / 3) ** 2 + (z - n / 2) ** 2 > (n / 5) ** 2) & (rng.random((n, n, n)) > 0.05)
    f = rng.normal(size=(3, n, n, n)).astype(np.float32)
    target = np.sin(x / 3.0) * np.cos(y / 4.0) + 0.1 * rng.normal(size=(n, n, n))
    return valid, f, target


def _params(seed):
    from paper_2311_16935_gb300 import seednet

    p = seednet.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    d = seednet.unpack(p)
    for k in d:
        if k.endswith(".b"):
            d[k][:] = rng.normal(size=d[k].shape) * 0.05
    return p, d


def _oracle_params(d):
    out = {}
    for k, v in d.items():
        out[k] = bf16_round(v) if k.endswith(".w") else np.asarray(v, dtype=np.float32).astype(np.float64)
    return out


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


@pytest.mark.parametrize("n", [16, 24])
def test_forward_matches_reference(osm, n):
    """The forward pass (tcgen05 tensor cores) element by element against the
    FP64 reference fed the same BF16 weights and input and storing every
    activation in BF16 as the GPU does: max |GPU - reference| <= 1e-2 of the
    output's largest magnitude.  Rounding the FP32-accumulated sums to BF16
    can land on the other side of a BF16 rounding boundary than the FP64
    sum; such flips are one BF16 ulp (2^-8 relative) of one activation and
    stay far below the bound after the remaining layers."""
    valid, f, target = _problem(n, 1)
    params, d = _params(2)
    net = osm.Net((n, n, n), train=False)
    net.set_params(params)
    g = torch.from_numpy(f).cuda()
    m = torch.from_numpy(valid.astype(np.uint8)).cuda()
    p = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    net.forward(g, m, 1.0, p)
    got = net.get_output()
    x, s = onet.features(f.astype(np.float64), valid, 1.0)
    want, _ = onet.forward(_oracle_params(d), bf16_round(x), store=bf16_round)
    scale = float(np.abs(want).max())
    assert float(np.abs(got - want).max()) <= 1e-2 * scale
    assert _rel(got, want) < 1e-2
    np.testing.assert_allclose(p.cpu().numpy()[valid], got[valid] * s, rtol=1e-5, atol=1e-6 * s)
    net.close()


def test_tcgen05_and_wmma_paths_agree(osm):
    """Forward output and every parameter gradient of the tcgen05 path
    against the warp-level wmma path (OSMODI_DEBUG_NET_WMMA) on the same
    inputs: the same BF16 products summed in FP32 in another order."""
    n = 32
    valid, f, target = _problem(n, 5)
    params, d = _params(6)
    g = torch.from_numpy(f).cuda()
    m = torch.from_numpy(valid.astype(np.uint8)).cuda()
    tgt = torch.from_numpy(target).cuda()
    outs = {}
    for wmma in (0, 1):
        osm.debug_set(osm.DEBUG_NET_WMMA, wmma)
        try:
            net = osm.Net((n, n, n), train=True)
            net.set_params(params)
            loss = net.backward(g, m, 1.0, tgt)
            outs[wmma] = (net.get_output(), net.get_grads(), loss)
            net.close()
        finally:
            osm.debug_set(osm.DEBUG_NET_WMMA, osm.DEBUG_DEFAULT)
    (o0, g0, l0), (o1, g1, l1) = outs[0], outs[1]
    assert float(np.abs(o0 - o1).max()) <= 1e-2 * float(np.abs(o1).max())
    assert l0 == pytest.approx(l1, rel=1e-2)
    from paper_2311_16935_gb300 import seednet

    d0, d1 = seednet.unpack(g0), seednet.unpack(g1)
    scale = max(float(np.abs(v).max()) for v in d1.values())
    for k in d1:
        a, b = np.ravel(d0[k]).astype(np.float64), np.ravel(d1[k]).astype(np.float64)
        if k == "out.b":  # exactly 0 (the loss ignores constants): compare absolutely
            assert abs(a[0]) <= 1e-5 * scale and abs(b[0]) <= 1e-5 * scale
            continue
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert _rel(a, b) < 5e-2 and cos > 0.998, (k, _rel(a, b), cos)


def test_parameter_gradients_match_reference(osm):
    """Parameter gradients against the FP64 reference fed the same BF16-stored
    activations and operands.  The remaining differences are FP32-vs-FP64
    accumulation flipping individual BF16 roundings (one BF16 ulp, 2^-8
    relative, of an activation whose sum lies within ~1e-6 of a rounding
    boundary; a flip can also flip a ReLU).  A weight gradient sums such
    errors over the voxels of its level, so its relative error grows as the
    level shrinks: on this 32^3 net the levels below half resolution hold 8^3
    and 4^3 voxels.  Bounds: 2e-2 (the survey's figure) at full and half
    resolution, 5e-2 at the two coarse levels (measured worst 3.5e-2, the
    4^3 bottleneck), every tensor pointing the same way (cosine >= 0.999)."""
    n = 32
    valid, f, target = _problem(n, 3)
    params, d = _params(4)
    net = osm.Net((n, n, n), train=True)
    net.set_params(params)
    g = torch.from_numpy(f).cuda()
    m = torch.from_numpy(valid.astype(np.uint8)).cuda()
    tgt = torch.from_numpy(target).cuda()
    loss = net.backward(g, m, 1.0, tgt)
    grads = net.get_grads()
    x, s = onet.features(f.astype(np.float64), valid, 1.0)
    op = _oracle_params(d)
    # the GPU stores activations and MMA operands in BF16: the reference
    # quantises the same stored values (so both take the same ReLU decisions)
    out, act = onet.forward(op, bf16_round(x), store=bf16_round)
    L, gl = onet.loss(out, target / s, valid)
    ref = onet.backward(op, act, gl, operand=bf16_round)
    assert loss == pytest.approx(L, rel=1e-2)
    from paper_2311_16935_gb300 import seednet

    gd = seednet.unpack(grads)
    scale = max(np.abs(v).max() for v in ref.values())
    level = {"e0": 0, "u0": 0, "out": 0, "e1": 1, "e1b": 1, "u1": 1, "u1b": 1}
    worst = {}
    for k in ref:
        if k == "out.b":  # exactly 0 (the loss ignores constants): compare absolutely
            assert abs(float(gd[k][0])) <= 1e-5 * scale, (gd[k], ref[k])
            continue
        a, b = np.ravel(gd[k]).astype(np.float64), np.ravel(ref[k])
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        worst[k] = (_rel(a, b), cos)
    print("gradient rel. error, cosine by tensor:", sorted(worst.items(), key=lambda kv: -kv[1][0]))
    bad = {k: v for k, v in worst.items()
           if v[0] > (2e-2 if level.get(k.split(".")[0], 2) <= 1 else 5e-2) or v[1] < 0.999}
    assert not bad, sorted(worst.items(), key=lambda kv: -kv[1][0])
    net.close()


def test_training_reduces_loss_and_seed_helps(osm):
    """Train on a few method-solved pairs at 32^3, then seed held-out solves:
    the guess starts closer than zero and the seeded plain-CG solve needs
    fewer iterations to the same tolerance.  With the multigrid
    preconditioner the iteration count hardly depends on the start (a
    V-cycle removes a fixed fraction of every error mode), so there the seed
    must cost no more than one iteration on average."""
    from paper_2311_16935_gb300 import seednet

    n = 32
    pairs = seednet.make_pairs(24, n, seed0=2000, tol=1e-9)
    params, hist = seednet.train(pairs, n, epochs=25, lr=2e-3, batch=4, seed=0)
    assert hist[-1] < 0.5 * hist[0], hist
    dists, saved = [], []
    for i in range(4):
        prob = seednet.blob_problem(n, 9000 + i)
        p, r_seed, r_zero = seednet.seeded_solve(params, prob.grad, n, 1e-9)
        assert r_seed.status == osm.OK and r_zero.status == osm.OK
        dists.append(r_seed.seed_rel_dist)
        saved.append(r_zero.inner_iters - r_seed.inner_iters)
    assert np.mean(dists) < 0.9, dists
    assert np.mean(saved) > 0, saved
    plan = osm.Plan(3, (n, n, n), (1.0, 1.0, 1.0), None, precision=osm.FP32_REFINE, precond=1)
    it_seed, it_zero = [], []
    for i in range(4):
        prob = seednet.blob_problem(n, 9000 + i)
        _, r_seed, r_zero = seednet.seeded_solve(params, prob.grad, n, 1e-9, plan=plan)
        assert r_seed.status == osm.OK and r_zero.status == osm.OK
        it_seed.append(r_seed.inner_iters)
        it_zero.append(r_zero.inner_iters)
    plan.close()
    assert np.mean(it_seed) <= np.mean(it_zero) + 1.0, (it_seed, it_zero)


@pytest.mark.parametrize("n", [64, 128, 256])
def test_forward_paths_agree_at_width(osm, n):
    """At the widths where the tensor-core kernels change tiling (rows of 64,
    one 128-voxel segment, two segments per row) the forward pass on tcgen05
    equals the wmma path's to BF16 rounding of the stored activations."""
    from paper_2311_16935_gb300 import seednet

    prob = seednet.blob_problem(n, 77)
    params = seednet.init_params(3)
    outs = []
    for wmma in (0, 1):
        osm.debug_set(osm.DEBUG_NET_WMMA, wmma)
        try:
            net = osm.Net((n, n, n), train=False)
            net.set_params(params)
            p = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
            net.forward(prob.grad, None, 1.0, p)
            outs.append(net.get_output())
            net.close()
        finally:
            osm.debug_set(osm.DEBUG_NET_WMMA, osm.DEBUG_DEFAULT)
    a, b = outs
    assert np.isfinite(a).all()
    assert float(np.abs(a - b).max()) <= 1e-2 * float(np.abs(b).max())
