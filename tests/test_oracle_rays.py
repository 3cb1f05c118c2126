"""Pins of eps_P (Eq. ResidualPressure) and the whole-ray check of Section
"Limit of Infinite Rays" (no GPU).

The method takes the rotating-parallel-ray integration to the limit of
infinitely many rays.  Whole straight rays at a finite density are averaged
and iterated here (oracle.rotating_ray_solve_2d) and compared with the fixed
point of Algorithm 1 (oracle.solve_direct): for fields whose face steps are
exact the two agree at any density; for a smooth field with noise the
distance shrinks as the ray density grows and the rays' error against the
true pressure approaches the matrix method's -- a trend check, not parity
(a straight ray carries its own value from cell to cell, where Algorithm 1
carries the cell's average over all rays, so the two limits differ by a
small amount on noisy data)."""
import math

import numpy as np
import pytest

import oracle
from paper_2311_16935_gb300 import inputs


def _rel(a, b, valid):
    return float(np.linalg.norm(a[valid] - b[valid]) / np.linalg.norm(b[valid]))


def test_pressure_update_hand_values():
    """eps_P = ||P^{n+1} - P^n|| / ||P^{n+1}|| over valid cells, by hand:
    P^{n+1} = (3, 4), P^n = (3, 1) gives 3 / 5 (the other denominator,
    ||P^n|| = sqrt(10), would give 0.9487); missing cells do not count."""
    valid = np.array([True, True, False])
    assert oracle.pressure_update([3.0, 4.0, 1e9], [3.0, 1.0, -7.0], valid) == pytest.approx(0.6, abs=1e-15)
    assert oracle.pressure_update([3.0, 1.0, 0.0], [3.0, 4.0, 0.0], valid) == pytest.approx(3 / math.sqrt(10), abs=1e-15)
    assert oracle.pressure_update([0.0, 0.0, 5.0], [1.0, 2.0, 5.0], valid) == 0.0
    # scale invariance, and eps_P = 1 from a zero start
    assert oracle.pressure_update([6.0, 8.0, 0.0], [6.0, 2.0, 0.0], valid) == pytest.approx(0.6, abs=1e-15)
    assert oracle.pressure_update([2.0, -1.0, 0.0], [0.0, 0.0, 0.0], valid) == 1.0


def test_literal_history_of_eps_P():
    """Algorithm 1's recorded eps_P: the first iteration from P^0 = 0 has
    eps_P = 1 exactly, and every later entry is ||P^{n+1} - P^n|| / ||P^{n+1}||
    of the iterates themselves (re-run step by step here with a different
    linear solver, dense inverse instead of sparse LU)."""
    rng = np.random.default_rng(4)
    valid = rng.random((7, 8)) > 0.15
    grid = oracle.Grid(valid, (0.1, 0.13))
    f = rng.normal(size=(2, 7, 8))
    _, n, er, ep = oracle.solve_literal(grid, f, tol=1e-6)
    assert ep[0] == 1.0
    W1, Wn = oracle.operators(grid)
    v = np.flatnonzero(valid.reshape(-1))
    M = (np.eye(grid.n) - W1.toarray())[np.ix_(v, v)]
    Wv = Wn.toarray()[np.ix_(v, v)]
    S = oracle.source(grid, f).reshape(-1)[v]
    Minv = np.linalg.inv(M)
    P = np.zeros(v.size)
    for k in range(min(n, 30)):
        Pn1 = Minv @ (Wv @ P + S)
        assert ep[k] == pytest.approx(np.linalg.norm(Pn1 - P) / np.linalg.norm(Pn1), rel=1e-9)
        P = Pn1


def test_whole_rays_recover_exact_steps():
    """A quadratic pressure with its exact gradient makes every face step of
    Eq. PressureIntegrator1 exact, so whole straight rays give the true
    pressure (up to a constant) at any ray density, as Algorithm 1 does."""
    shape, spacing = (9, 11), (0.1, 0.13)
    p, g = inputs.quadratic_field(shape, spacing, seed=5)
    p, g = p.numpy(), g.numpy()
    valid = np.ones(shape, bool)
    valid[3:5, 4:7] = False
    grid = oracle.Grid(valid, spacing)
    want = oracle.gauge(grid, p)
    for n_theta, ds in ((12, 0.06), (40, 0.03)):
        P, it = oracle.rotating_ray_solve_2d(grid, g, n_theta, ds)
        assert _rel(P, want, valid) < 1e-10, (n_theta, ds)
    assert _rel(oracle.solve_direct(grid, g), want, valid) < 1e-12


def test_whole_rays_approach_the_fixed_point():
    """Gaussian pressure bump with 1 % gradient noise on a 13 x 13 grid with a
    hole: at three ray densities the distance between the iterated whole-ray
    average and Algorithm 1's fixed point falls monotonically, and the rays'
    error against the true pressure approaches the fixed point's (the
    behaviour of Figure InfiniteRays)."""
    n = 13
    h = 1.0 / (n - 1)
    y, x = np.meshgrid(np.arange(n) * h, np.arange(n) * h, indexing="ij")
    w = 0.05
    p = np.exp(-((x - 0.5) ** 2 + (y - 0.5) ** 2) / w)
    g = np.stack([-2 * (x - 0.5) / w * p, -2 * (y - 0.5) / w * p])
    g = g + 0.01 * np.abs(g).max() * np.random.default_rng(7).normal(size=g.shape)
    valid = np.ones((n, n), bool)
    valid[6:8, 3:5] = False
    grid = oracle.Grid(valid, (h, h))
    P_fix = oracle.solve_direct(grid, g)
    truth = oracle.gauge(grid, p)
    e_fix = _rel(P_fix, truth, valid)
    dist, gap = [], []
    for n_theta, ds in ((12, 0.6 * h), (40, 0.25 * h), (120, 0.1 * h)):
        P, it = oracle.rotating_ray_solve_2d(grid, g, n_theta, ds)
        assert it < 100000
        dist.append(_rel(P, P_fix, valid))
        gap.append(abs(_rel(P, truth, valid) - e_fix))
    assert dist[0] > dist[1] > dist[2], dist
    assert dist[2] < 0.5 * dist[0] and dist[2] < 5e-3, dist
    assert gap[2] < gap[0] and gap[2] < 0.05 * e_fix, (gap, e_fix)
