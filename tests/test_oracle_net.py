"""Pins of the CPU reference of the seed network: every layer's backward and
the whole model's gradient against central finite differences (no GPU)."""
import numpy as np
import pytest

from oracle import net


def _fd_check(f, x, g_analytic, n_probe=12, h=1e-5, seed=0):
    """Compare directional derivatives along random directions."""
    rng = np.random.default_rng(seed)
    for _ in range(n_probe):
        d = rng.normal(size=x.shape)
        fp = f(x + h * d)
        fm = f(x - h * d)
        num = (fp - fm) / (2 * h)
        ana = float((g_analytic * d).sum())
        assert abs(num - ana) <= 1e-6 * max(1.0, abs(ana)), (num, ana)


@pytest.mark.parametrize("kind,shape,cin,cout", [("conv3", (4, 5, 6), 3, 5), ("down", (4, 6, 8), 3, 4),
                                                 ("up", (2, 3, 4), 4, 3), ("conv1", (3, 3, 4), 5, 2)])
def test_layer_backward(kind, shape, cin, cout):
    rng = np.random.default_rng(1)
    x = rng.normal(size=shape + (cin,))
    w = rng.normal(size=(net.TAPS[kind], cin, cout))
    b = rng.normal(size=cout)
    fwd, bwd = net._FWD[kind], net._BWD[kind]
    y = fwd(x, w, b)
    r = rng.normal(size=y.shape)  # random linear functional L = <r, y>
    dx, dw, db = bwd(x, w, r)
    _fd_check(lambda xx: float((fwd(xx, w, b) * r).sum()), x, dx)
    _fd_check(lambda ww: float((fwd(x, ww, b) * r).sum()), w, dw)
    _fd_check(lambda bb: float((fwd(x, w, bb) * r).sum()), b, db)


def test_layer_definitions_by_brute_force():
    """conv3 / down / up written as explicit loops over voxels and taps."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=(4, 4, 4, 2))
    w = rng.normal(size=(27, 2, 3))
    y = net.conv3(x, w, np.zeros(3))
    z, yy, xx = 1, 2, 0
    ref = np.zeros(3)
    t = 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                iz, iy, ix = z + dz, yy + dy, xx + dx
                if 0 <= iz < 4 and 0 <= iy < 4 and 0 <= ix < 4:
                    ref += x[iz, iy, ix] @ w[t]
                t += 1
    np.testing.assert_allclose(y[z, yy, xx], ref, rtol=1e-13)
    w8 = rng.normal(size=(8, 2, 3))
    d = net.down(x, w8, np.zeros(3))
    ref = sum(x[2 * 1 + pz, 2 * 0 + py, 2 * 1 + px] @ w8[pz * 4 + py * 2 + px]
              for pz in (0, 1) for py in (0, 1) for px in (0, 1))
    np.testing.assert_allclose(d[1, 0, 1], ref, rtol=1e-13)
    u = net.up(d, w8.transpose(0, 2, 1).copy(), np.zeros(2))
    np.testing.assert_allclose(u[3, 0, 2], d[1, 0, 1] @ w8[4 + 0 + 0].T, rtol=1e-13)


def test_model_gradient_finite_differences():
    rng = np.random.default_rng(3)
    params = net.init_params(seed=4)
    # nonzero biases so that every ReLU pattern is exercised
    for k in params:
        if k.endswith(".b"):
            params[k] = rng.normal(size=params[k].shape) * 0.1
    x = rng.normal(size=(8, 8, 8, 4))
    valid = rng.random((8, 8, 8)) > 0.2
    target = rng.normal(size=(8, 8, 8))

    def L_of(p):
        out, _ = net.forward(p, x)
        return net.loss(out, target, valid)[0]

    out, act = net.forward(params, x)
    L, g = net.loss(out, target, valid)
    grads = net.backward(params, act, g)
    for key in ["e0.w", "e1.b", "m.w", "u2.w", "u0.w", "out.w", "out.b", "e2b.w"]:
        base = params[key]

        def f(v, key=key):
            q = dict(params)
            q[key] = v
            return L_of(q)

        _fd_check(f, base, grads[key], n_probe=4, h=1e-6)


def test_loss_is_gauge_invariant():
    rng = np.random.default_rng(5)
    out = rng.normal(size=(4, 4, 4))
    tgt = rng.normal(size=(4, 4, 4))
    valid = rng.random((4, 4, 4)) > 0.3
    L1, g1 = net.loss(out, tgt, valid)
    L2, g2 = net.loss(out + 3.0, tgt - 1.0, valid)
    assert L1 == pytest.approx(L2, rel=1e-12)
    np.testing.assert_allclose(g1, g2, atol=1e-14)
    assert abs(g1[valid].sum()) < 1e-12
