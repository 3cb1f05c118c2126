"""Pins of the front-end oracle (no GPU): the difference rule against
analytic derivatives, closed-form flows whose pressure is known exactly, and
second-order convergence on exact solutions of the flow equations."""
import numpy as np
import pytest

import oracle
from oracle import front


def _grid2(nx, ny, hx, hy):
    y, x = np.meshgrid(np.arange(ny) * hy, np.arange(nx) * hx, indexing="ij")
    return x, y


def _random_mask(shape, seed, drop=0.2):
    rng = np.random.default_rng(seed)
    return rng.random(shape) > drop


def _has_axis_neighbour(valid, a):
    ax = valid.ndim - 1 - a
    vp = np.zeros_like(valid)
    vm = np.zeros_like(valid)
    sl = lambda lo, hi: tuple(slice(lo, hi) if d == ax else slice(None) for d in range(valid.ndim))
    vp[sl(0, -1)] = valid[sl(1, None)]
    vm[sl(1, None)] = valid[sl(0, -1)]
    return valid & (vp | vm)


def _holes_mask(x, y, holes):
    valid = np.ones(x.shape, bool)
    for cx, cy, r in holes:
        valid &= (x - cx) ** 2 + (y - cy) ** 2 > r * r
    return valid


def test_difference_rule_exact_on_polynomials():
    """Linear fields: every case of the first-derivative rule is exact.
    Quadratic fields: the centred and three-point one-sided cases (all that a
    full grid uses) are exact for both derivatives."""
    hx, hy = 0.1, 0.13
    x, y = _grid2(17, 12, hx, hy)
    valid = _random_mask(x.shape, 1, drop=0.3)
    lin = 0.3 + 1.7 * x - 2.2 * y
    for a, h, slope in ((0, hx, 1.7), (1, hy, -2.2)):
        d = front.d1(lin, valid, a, h)
        has = _has_axis_neighbour(valid, a)
        np.testing.assert_allclose(d[has], slope, rtol=1e-11)
        assert np.all(d[valid & ~has] == 0.0)
    full = np.ones_like(valid)
    q = 0.5 + x - 3 * y + 2 * x * x - 1.5 * x * y + 0.7 * y * y
    np.testing.assert_allclose(front.d1(q, full, 0, hx), 1 + 4 * x - 1.5 * y, rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(front.d1(q, full, 1, hy), -3 - 1.5 * x + 1.4 * y, rtol=1e-10, atol=1e-11)
    np.testing.assert_allclose(front.d2(q, full, 0, hx), 4.0, rtol=1e-9)
    np.testing.assert_allclose(front.d2(q, full, 1, hy), 1.4, rtol=1e-9)
    # on a masked grid the quadratic is exact wherever a 3-point rule applied
    d = front.d1(q, valid, 0, hx)
    vp = np.zeros_like(valid); vp[:, :-1] = valid[:, 1:]
    vm = np.zeros_like(valid); vm[:, 1:] = valid[:, :-1]
    vpp = np.zeros_like(valid); vpp[:, :-2] = valid[:, 2:]
    vmm = np.zeros_like(valid); vmm[:, 2:] = valid[:, :-2]
    three = valid & ((vp & vm) | (vp & vpp) | (~vp & vm & vmm))
    assert three.sum() > 0.5 * valid.sum()
    np.testing.assert_allclose(d[three], (1 + 4 * x - 1.5 * y)[three], rtol=1e-10, atol=1e-11)
    # isolated along the axis: 0
    lone = valid & ~vp & ~vm
    assert np.all(d[lone] == 0.0)


def test_difference_rule_3d_axes():
    n = 9
    z, y, x = np.meshgrid(*[np.arange(n) * 0.2] * 3, indexing="ij")
    full = np.ones((n, n, n), bool)
    q = x * x + 2 * y * z - z
    np.testing.assert_allclose(front.d1(q, full, 0, 0.2), 2 * x, atol=1e-11)
    np.testing.assert_allclose(front.d1(q, full, 1, 0.2), 2 * z, atol=1e-11)
    np.testing.assert_allclose(front.d1(q, full, 2, 0.2), 2 * y - 1, atol=1e-11)
    np.testing.assert_allclose(front.d2(q, full, 0, 0.2), 2.0, atol=1e-9)


@pytest.mark.parametrize("flow", ["rotation", "stagnation"])
def test_rans_linear_mean_flows_recover_exact_pressure(flow):
    """Steady inviscid flows with linear velocity: solid-body rotation
    (p = rho W^2 r^2 / 2) and plane stagnation flow (p = -rho a^2 (x^2 +
    y^2) / 2).  Every difference is exact, so the source equals grad p, and
    the integration (quadratic pressure: an exact fixed point) returns p up
    to a constant, on a masked grid."""
    hx, hy, rho = 0.05, 0.07, 1.3
    x, y = _grid2(21, 16, hx, hy)
    # PIV-like solid bodies, clear of the edges: no cell lacks both
    # neighbours along an axis (there the rule has no derivative to offer)
    valid = _holes_mask(x, y, [(0.3, 0.4, 0.16), (0.72, 0.68, 0.17)])
    for a in (0, 1):
        assert np.array_equal(_has_axis_neighbour(valid, a), valid)
    xc, yc = 0.5, 0.5
    if flow == "rotation":
        w = 2.0
        U = np.stack([-w * (y - yc), w * (x - xc)])
        p = rho * w * w * ((x - xc) ** 2 + (y - yc) ** 2) / 2
    else:
        a = 1.5
        U = np.stack([a * (x - xc), -a * (y - yc)])
        p = -rho * a * a * ((x - xc) ** 2 + (y - yc) ** 2) / 2
    R = np.zeros((3,) + x.shape)
    f = front.rans(valid, (hx, hy), U, R, rho=rho)
    g = np.stack([np.gradient(p, hx, axis=1), np.gradient(p, hy, axis=0)])  # exact for quadratics inside
    inner = valid.copy()
    inner[:, [0, -1]] = False
    inner[[0, -1], :] = False
    for i in range(2):
        np.testing.assert_allclose(f[i][inner], g[i][inner], rtol=1e-10, atol=1e-10)
    grid = oracle.Grid(valid, (hx, hy))
    P = oracle.solve_direct(grid, f)
    want = oracle.gauge(grid, np.where(valid, p, np.nan))
    assert np.linalg.norm(P[valid] - want[valid]) <= 1e-9 * np.linalg.norm(want[valid])


def test_reynolds_stress_divergence_exact_for_quadratics():
    hx, hy = 0.1, 0.1
    x, y = _grid2(14, 11, hx, hy)
    full = np.ones(x.shape, bool)
    U = np.zeros((2,) + x.shape)
    R = np.stack([x * x, y * y, x * y])  # xx, yy, xy
    f = front.rans(full, (hx, hy), U, R, rho=2.0)
    # d/dx xx + d/dy xy = 2x + x ; d/dx xy + d/dy yy = y + 2y
    np.testing.assert_allclose(f[0], -2.0 * 3 * x, atol=1e-10)
    np.testing.assert_allclose(f[1], -2.0 * 3 * y, atol=1e-10)


def _taylor_green(n, nu=0.05, rho=1.0, t=0.3, dt=1e-3):
    h = 2 * np.pi / n
    x, y = _grid2(n, n, h, h)
    F = lambda tt: np.exp(-2 * nu * tt)

    def vel(tt):
        return np.stack([np.cos(x) * np.sin(y) * F(tt), -np.sin(x) * np.cos(y) * F(tt)])

    p = -rho / 4 * (np.cos(2 * x) + np.cos(2 * y)) * F(t) ** 2
    gp = np.stack([rho / 2 * np.sin(2 * x) * F(t) ** 2, rho / 2 * np.sin(2 * y) * F(t) ** 2])
    return h, vel(t - dt), vel(t), vel(t + dt), dt, p, gp, rho, rho * nu


def test_incompressible_second_order_on_taylor_green():
    """The Taylor-Green vortex solves the incompressible Navier-Stokes
    equations exactly; the source of Eq. 1 built from three snapshots
    converges to grad p at second order, and so does the integrated pressure."""
    errs, perrs = [], []
    for n in (24, 48, 96):
        h, um, u0, up, dt, p, gp, rho, mu = _taylor_green(n)
        valid = np.ones(u0.shape[1:], bool)
        f = front.incompressible(valid, (h, h), u0, um, up, dt=dt, rho=rho, mu=mu)
        # away from the edges (where the one-sided second difference is
        # first order) the source is second order
        errs.append(np.abs(f - gp)[:, 2:-2, 2:-2].max() / np.abs(gp).max())
        grid = oracle.Grid(valid, (h, h))
        P = oracle.solve_cg(grid, f, tol=1e-13)[0]
        want = oracle.gauge(grid, p)
        perrs.append(np.abs(P - want).max() / np.abs(want).max())
    for e in (errs, perrs):
        assert e[0] / e[1] > 3.2 and e[1] / e[2] > 3.2, e


def test_uniform_and_still_flows_have_no_source():
    shape = (6, 7, 8)
    valid = _random_mask(shape, 5)
    U = np.stack([np.full(shape, 3.0), np.full(shape, -1.0), np.full(shape, 0.5)])
    R = np.stack([np.full(shape, v) for v in (0.1, 0.2, 0.3, 0.01, 0.02, 0.03)])
    assert np.abs(front.incompressible(valid, (1, 1, 1), U, mu=0.3)).max() < 1e-12
    assert np.abs(front.rans(valid, (1, 1, 1), U, R)).max() < 1e-12
    g, _ = front.compressible(valid, (1, 1, 1), U, R, 1.4, 0.5, 3.5, 300.0, 287.0)
    assert np.abs(g).max() < 1e-15


def _compressible_1d(n, theta, a_stress):
    """A steady inviscid 1D flow along e = (cos theta, sin theta): the
    conservative momentum balance d/ds(rho <u u>) + dP/ds = 0 with rho =
    P/(R T) gives P (1 + <u_s u_s>/(R T)) = const for any temperature
    profile, so ln(P/P_inf) = const - ln(1 + <u_s u_s>/(R T))."""
    gamma, mach, vinf, tinf, rgas = 1.4, 0.6, 200.0, 280.0, 287.0
    L = 1.0
    h = L / (n - 1)
    x, y = _grid2(n, n, h, h)
    e = np.array([np.cos(theta), np.sin(theta)])
    s = e[0] * x + e[1] * y
    q = vinf * (1.0 + 0.3 * np.sin(2.0 * np.pi * s / L))  # total <u_s u_s> = q^2
    Um = np.sqrt(1.0 - a_stress) * q
    U = np.stack([Um * e[0], Um * e[1]])
    rs = a_stress * q * q
    R = np.stack([rs * e[0] * e[0], rs * e[1] * e[1], rs * e[0] * e[1]])
    T = front.temperature(U, gamma, mach, vinf, tinf)
    lnp = -np.log(1.0 + q * q / (rgas * T))
    return h, U, R, (gamma, mach, vinf, tinf, rgas), lnp


@pytest.mark.parametrize("theta,a_stress", [(0.0, 0.0), (0.6, 0.0), (0.6, 0.3)])
def test_compressible_closed_form_second_order(theta, a_stress):
    errs = []
    for n in (21, 41, 81):
        h, U, R, consts, lnp = _compressible_1d(n, theta, a_stress)
        valid = np.ones(lnp.shape, bool)
        g, _ = front.compressible(valid, (h, h), U, R, *consts)
        grid = oracle.Grid(valid, (h, h))
        P = oracle.solve_cg(grid, g, tol=1e-13)[0]
        want = oracle.gauge(grid, lnp)
        errs.append(np.abs(P - want).max() / np.abs(want).max())
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs
    assert errs[2] < 5e-3


def test_compressible_reduces_to_rans_at_low_speed():
    """With M_inf = 0 (T = T_inf) and U -> 0, (I + <u u>/(R T)) -> I and
    R T g -> -d<u_i u_j>/dx_j, the momentum-flux divergence per unit
    density.  For linear U and quadratic stresses on a full grid every
    difference is exact, so the product rule holds discretely:
    -d(U_i U_j + R_ij)/dx_j = f_RANS,i - U_i div U."""
    n = 15
    h = 0.1
    x, y = _grid2(n, n, h, h)
    full = np.ones(x.shape, bool)
    eps = 1e-4
    U = eps * np.stack([0.3 + 1.2 * x - 0.7 * y, -0.2 + 0.4 * x + 0.9 * y])
    R = eps * eps * np.stack([x * x, y * y, 0.1 * x * y])
    tinf, rgas = 300.0, 287.0
    g, T = front.compressible(full, (h, h), U, R, 1.4, 0.0, 1.0, tinf, rgas)
    assert np.all(T == tinf)
    f = front.rans(full, (h, h), U, R, rho=1.0)
    divU = eps * (1.2 + 0.9)
    np.testing.assert_allclose(rgas * tinf * g, f - U * divU, rtol=1e-9, atol=1e-12 * np.abs(f).max())


def test_compressible_3d_pointwise_second_order():
    """The closed-form 1D flow along a 3D diagonal (the 3 x 3 system with
    all cross terms): grad ln(P/P_inf) from the oracle converges to the
    analytic gradient at second order away from the edges."""
    gamma, mach, vinf, tinf, rgas, a_st = 1.4, 0.6, 200.0, 280.0, 287.0, 0.25
    e = np.array([0.5, 0.6, np.sqrt(1.0 - 0.61)])
    c = 0.5 * (gamma - 1.0) * mach ** 2
    k = 2.0 * np.pi
    errs = []
    for n in (10, 20, 40):
        h = 1.0 / (n - 1)
        z, y, x = np.meshgrid(*[np.arange(n) * h] * 3, indexing="ij")
        s = e[0] * x + e[1] * y + e[2] * z
        q = vinf * (1.0 + 0.3 * np.sin(k * s))
        dq = vinf * 0.3 * k * np.cos(k * s)
        Um = np.sqrt(1.0 - a_st) * q
        U = np.stack([Um * e[0], Um * e[1], Um * e[2]])
        rs = a_st * q * q
        R = np.stack([rs * e[0] * e[0], rs * e[1] * e[1], rs * e[2] * e[2],
                      rs * e[0] * e[1], rs * e[0] * e[2], rs * e[1] * e[2]])
        T = tinf * (1.0 + c * (1.0 - (1.0 - a_st) * q * q / vinf ** 2))
        dT = -tinf * c * (1.0 - a_st) * 2.0 * q * dq / vinf ** 2
        w = q * q / (rgas * T)
        dw = (2.0 * q * dq * T - q * q * dT) / (rgas * T * T)
        dphi = -dw / (1.0 + w)
        g, Tg = front.compressible(np.ones(x.shape, bool), (h, h, h), U, R, gamma, mach, vinf, tinf, rgas)
        np.testing.assert_allclose(Tg, T, rtol=1e-12)
        sl = (slice(None),) + (slice(2, -2),) * 3
        want = np.stack([dphi * e[0], dphi * e[1], dphi * e[2]])
        errs.append(np.abs(g - want)[sl].max() / np.abs(want).max())
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.5, errs
